// The C ABI and the host-side driver of the augmented subspace iteration.
//
// pase_setup builds the device data (paper §3 Alg. 3 "Require": A_h, B_h = M_h, the
// interpolation chain I_H^h, A_H, B_H); pase_solve runs Alg. 2 / Alg. 3 with one
// "Correction" (Alg. 1) per outer iteration:
//   residual   R = M U Lambda - A U, relative residuals            (convergence test, §6)
//   (a)        W = U + V-cycles(R)  [FP64, or FP32 inside FP64 refinement]  (Alg. 3 step 3)
//   (b)        aH = P^T A W, bH = P^T M W, GA = W^T A W, GM = W^T M W      (Alg. 3 step 4)
//   (c)        m smallest pairs of the augmented pencil, warm start u_H = 0, gamma = I
//              (Alg. 3 step 5; solved by a block eigensolver in the spirit of GCG_AUG,
//              Alg. 4, with a preconditioner built from the PRECOND-A factors of §4)
//   (d)        U = P C_H + W C_W                                             (Alg. 3 step 6)
// Every arithmetic step is a kernel of this library; the host only sequences launches and
// reads back m residual norms per iteration.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <array>
#include <memory>
#include <mutex>
#include <thread>

#include "pase_internal.h"

namespace pase {
const char* last_error_cstr();

int dev_alloc(pase_ctx* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? PASE_ERR_OUT_OF_MEMORY : PASE_ERR_CUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  h->allocations.push_back(*p);
  return PASE_OK;
}

int upload_csr(pase_ctx* h, const HostCSR& a, DevCSR& d, bool with_fp32, bool share,
               const DevCSR* src) {
  d.nrows = a.nrows;
  d.ncols = a.ncols;
  d.nnz = a.nnz();
  if (share && src) {
    d.rowptr = src->rowptr;
    d.col = src->col;
  } else {
    PASE_TRY(dev_alloc_t(h, &d.rowptr, a.nrows + 1));
    PASE_TRY(dev_alloc_t(h, &d.col, std::max<int64_t>(1, a.nnz())));
    PASE_CUDA(cudaMemcpy(d.rowptr, a.rowptr.data(), sizeof(int64_t) * (a.nrows + 1), cudaMemcpyHostToDevice));
    if (a.nnz()) PASE_CUDA(cudaMemcpy(d.col, a.col.data(), sizeof(int32_t) * a.nnz(), cudaMemcpyHostToDevice));
  }
  PASE_TRY(dev_alloc_t(h, &d.val, std::max<int64_t>(1, a.nnz())));
  if (a.nnz()) PASE_CUDA(cudaMemcpy(d.val, a.val.data(), sizeof(double) * a.nnz(), cudaMemcpyHostToDevice));
  if (with_fp32) {
    std::vector<float> v32(a.val.begin(), a.val.end());
    PASE_TRY(dev_alloc_t(h, &d.val32, std::max<int64_t>(1, a.nnz())));
    if (a.nnz()) PASE_CUDA(cudaMemcpy(d.val32, v32.data(), sizeof(float) * a.nnz(), cudaMemcpyHostToDevice));
  }
  return PASE_OK;
}

template <typename T>
static int upload_vec(pase_ctx* h, const std::vector<T>& v, T** d) {
  PASE_TRY(dev_alloc_t(h, d, std::max<size_t>(1, v.size())));
  if (!v.empty()) PASE_CUDA(cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return PASE_OK;
}

// ------------------------------------------------------------------ pointer staging
// Inputs/outputs of the ABI may be host or device memory; host ones go through a
// device staging buffer owned by the handle.
static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Stage {
  pase_ctx* h;
  std::vector<std::pair<void*, std::pair<void*, size_t>>> outs;  // (dev, (host, bytes))
  std::vector<size_t> taken;                                     // pool entries in use
  explicit Stage(pase_ctx* hh) : h(hh) {}
  ~Stage() {
    for (size_t i : taken) h->stage_pool[i].busy = false;
  }
  // a device buffer of at least `bytes` from the handle's pool (allocated on first need)
  int take(size_t bytes, void** out) {
    bytes = std::max<size_t>(bytes, 16);
    size_t best = SIZE_MAX;
    for (size_t i = 0; i < h->stage_pool.size(); ++i) {
      const auto& b = h->stage_pool[i];
      if (!b.busy && b.bytes >= bytes && (best == SIZE_MAX || b.bytes < h->stage_pool[best].bytes)) best = i;
    }
    if (best == SIZE_MAX) {
      void* p = nullptr;
      PASE_TRY(dev_alloc(h, &p, bytes));
      h->stage_pool.push_back({p, bytes, false});
      best = h->stage_pool.size() - 1;
    }
    h->stage_pool[best].busy = true;
    taken.push_back(best);
    *out = h->stage_pool[best].p;
    return PASE_OK;
  }
  // device view of an input
  int in(const void* p, size_t bytes, const void** dev) {
    if (!p) {
      *dev = nullptr;
      return PASE_OK;
    }
    if (is_device_ptr(p)) {
      *dev = p;
      return PASE_OK;
    }
    void* t = nullptr;
    PASE_TRY(take(bytes, &t));
    PASE_CUDA(cudaMemcpyAsync(t, p, bytes, cudaMemcpyHostToDevice, h->stream));
    *dev = t;
    return PASE_OK;
  }
  // device view of an output (copied back by finish()); inout copies in as well
  int out(void* p, size_t bytes, void** dev, bool inout = false) {
    if (!p) {
      *dev = nullptr;
      return PASE_OK;
    }
    if (is_device_ptr(p)) {
      *dev = p;
      return PASE_OK;
    }
    void* t = nullptr;
    PASE_TRY(take(bytes, &t));
    if (inout) PASE_CUDA(cudaMemcpyAsync(t, p, bytes, cudaMemcpyHostToDevice, h->stream));
    outs.push_back({t, {p, bytes}});
    *dev = t;
    return PASE_OK;
  }
  int finish() {
    for (auto& o : outs)
      PASE_CUDA(cudaMemcpyAsync(o.second.first, o.first, o.second.second, cudaMemcpyDeviceToHost, h->stream));
    PASE_CUDA(cudaStreamSynchronize(h->stream));
    return PASE_OK;
  }
};

// ------------------------------------------------------------------ live kernel timing
constexpr size_t kProfMaxLaunches = 4096;
void prof_begin(pase_ctx* h, int id) {
  if (id < 0 || id != h->prof_kernel || h->prof_n >= kProfMaxLaunches || recording(h)) return;
  while (h->prof_ev.size() < 2 * (h->prof_n + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    h->prof_ev.push_back(e);
  }
  cudaEventRecord(h->prof_ev[2 * h->prof_n], h->stream);
}
void prof_end(pase_ctx* h, int id) {
  if (id < 0 || id != h->prof_kernel || h->prof_n >= kProfMaxLaunches || h->prof_ev.size() < 2 * (h->prof_n + 1) ||
      recording(h))
    return;
  cudaEventRecord(h->prof_ev[2 * h->prof_n + 1], h->stream);
  h->prof_n++;
}

// ------------------------------------------------------------------ autotuner
// Threads of the small eigensolver's single-CTA stages (256, 512 or 1024), the form of
// its tridiagonalisation (one CTA, or a cluster of 8 or 16 SMs) and of its Cholesky
// factorisation (one CTA or a cluster of 8 SMs) for the three sizes the step-(c) block
// eigensolver uses (n = m, 2m, 3m; k = m): timed on a synthetic Gram pair, once per (n, k)
// in the process.
static int tune_sygv(pase_ctx* h) {
  Work& w = h->w;
  const int m = w.m, m3 = 3 * m;
  const int64_t nc = h->NH + m;
  if (w.aug_dense || nc < m3) return PASE_OK;  // the iterative step (c) does not run
  static std::mutex mu;
  // (n, k, fixed tridiagonalisation form, fixed Cholesky form; threads, forms chosen)
  static std::vector<std::array<int, 7>> cache;
  const int ftri = h->opt.sygv_tridiag, fch = h->opt.sygv_cholesky;
  PASE_TRY(launch_hash_fill(h, nc, m3, m3, 10u, w.S));
  PASE_TRY(launch_hash_fill(h, nc, m3, m3, 11u, w.AS));
  PASE_TRY(ts_gram(h, nc, m3, m3, w.AS, m3, w.AS, m3, w.Gq, m3, true));
  PASE_TRY(ts_gram(h, nc, m3, m3, w.S, m3, w.S, m3, w.Gb, m3, true));
  cudaEvent_t e0, e1;
  PASE_CUDA(cudaEventCreate(&e0));
  PASE_CUDA(cudaEventCreate(&e1));
  int rc = PASE_OK;
  for (int i = 0; i < 3 && rc == PASE_OK; ++i) {
    const int n = (i + 1) * m;
    h->sygv_n[i] = n;
    int found = 0, found_cl = -1, found_ch = -1;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (const auto& c : cache)
        if (c[0] == n && c[1] == m && c[2] == ftri && c[3] == fch) {
          found = c[4];
          found_cl = c[5];
          found_ch = c[6];
        }
    }
    if (found) {
      h->sygv_thr[i] = found;
      h->sygv_cl[i] = found_cl;
      h->sygv_ch[i] = found_ch;
      continue;
    }
    float best = 1e30f;
    int best_thr = 1024, best_cl = -1, best_ch = -1;
    for (int cand = 0; cand < 18; ++cand) {
      const int thr = (cand % 3 == 0) ? 1024 : (cand % 3 == 1 ? 512 : 256);
      const int cl = (cand / 3) % 3, ch = cand / 9;
      if (thr < m || ((cl || ch) && n < 16) || (cl == 2 && n < kTri16Min)) continue;
      if ((ftri >= 0 && cl != ftri) || (fch >= 0 && ch != fch)) continue;
      h->sygv_thr[i] = thr;
      h->sygv_cl[i] = cl;
      h->sygv_ch[i] = ch;
      for (int rep = 0; rep < 2 && rc == PASE_OK; ++rep) {
        if (rep == 1) rc = cudaEventRecord(e0, h->stream) == cudaSuccess ? PASE_OK : PASE_ERR_CUDA;
        for (int it = 0; it < 2 && rc == PASE_OK; ++it)
          rc = small_sygv(h, n, m, w.Gq, m3, w.Gb, m3, w.smallvec, w.Cs, m, w.status);
      }
      if (rc != PASE_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = fail(PASE_ERR_CUDA, "tune_sygv: event timing failed");
        break;
      }
      static const char* tri_form[3] = {"one-CTA", "8-SM cluster", "16-SM cluster"};
      if (h->opt.verbose >= 2)
        fprintf(stderr, "[pase]   small eigensolver n %d: %d threads, %s tridiagonalisation, %s Cholesky %.4f ms\n",
                n, thr, tri_form[cl], ch ? "8-SM cluster" : "one-CTA", ms / 2);
      if (ms < best) {
        best = ms;
        best_thr = thr;
        best_cl = cl;
        best_ch = ch;
      }
    }
    h->sygv_thr[i] = best_thr;
    h->sygv_cl[i] = best_cl;
    h->sygv_ch[i] = best_ch;
    if (h->opt.verbose)
      fprintf(stderr, "[pase] autotune small eigensolver n %d: %d threads, tridiagonalisation form %d, Cholesky "
              "form %d\n", n, best_thr, best_cl, best_ch);
    std::lock_guard<std::mutex> lk(mu);
    cache.push_back({n, m, ftri, fch, best_thr, best_cl, best_ch});
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// For every multigrid matrix, time the damped-Jacobi sweep (the precision the linear solve
// runs in) under each candidate schedule and keep the fastest: the CSR kernel at 128, 256
// and 512 threads per block and, for FP32 sweeps on a level the structured kernel serves,
// that kernel with one or two resident CTAs per SM, 3, 6 or 12 work items (plane chunks)
// per resident CTA, and 4 or 2 columns per consumer thread.  Deterministic operands; a few launches each, once per handle
// and block width.
static int autotune(pase_ctx* h) {
  Work& w = h->w;
  const int m = w.m;
  const bool mixed = h->opt.precision == PASE_PREC_MIXED;
  cudaEvent_t e0, e1;
  PASE_CUDA(cudaEventCreate(&e0));
  PASE_CUDA(cudaEventCreate(&e1));
  const int cand[3] = {128, 256, 512};
  for (int l = 0; l + 1 < h->L; ++l) {
    Level& L = h->lv[l];
    const int64_t nl = L.A.nrows;
    double *x = (l == 0) ? w.W : w.lx[l], *b = (l == 0) ? w.R : w.lb[l], *y = (l == 0) ? w.T1 : w.lt1[l];
    PASE_TRY(launch_hash_fill(h, nl, m, m, 3u, x));
    PASE_TRY(launch_hash_fill(h, nl, m, m, 4u, b));
    float *xf = nullptr, *bf = nullptr, *yf = nullptr;
    if (mixed) {
      xf = w.fx[l];
      bf = w.fb[l];
      yf = w.ft1[l];
      PASE_TRY(launch_f64_to_f32(h, nl * m, x, xf));
      PASE_TRY(launch_f64_to_f32(h, nl * m, b, bf));
    }
    float best = 1e30f;
    int best_bs = 256, best_use = 0, best_psm = 0, best_items = 6, best_cw = 4;
    // candidates: (structured kernel?, threads per block or CTAs per SM, items per CTA)
    struct Cand {
      int use, bs, psm, items, cw;
    };
    std::vector<Cand> cands;
    const int fixed_cw = h->opt.stencil_columns;  // 0: the autotuner chooses
    for (int c : cand) cands.push_back({0, c, 0, 6, fixed_cw ? fixed_cw : 4});
    const bool st =
        mixed && h->opt.stencil && L.A.st_val && h->tc_err && stencil_ok(L.A, CSR_JACOBI, m, 0, 0, h->opt.omega);
    if (st) {
      if (fixed_cw != 2)
        for (int psm : {2, 1})
          for (int items : {3, 6, 12}) cands.push_back({1, 256, psm, items, 4});
      if (fixed_cw != 4 && 16 * (m / 2) + 32 <= 512)
        for (int items : {3, 6, 12}) cands.push_back({1, 256, 2, items, 2});
    }
    for (const Cand& cd : cands) {
      L.A.block = cd.bs;
      L.A.st_use = cd.use;
      L.A.st_per_sm = cd.psm;
      L.A.st_items = cd.items;
      L.A.st_cw = cd.cw;
      for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) PASE_CUDA(cudaEventRecord(e0, h->stream));
        for (int it = 0; it < 3; ++it) {
          if (mixed)
            PASE_TRY(launch_csr<float>(h, CSR_JACOBI, m, L.A, L.A.val32, nullptr, xf, nullptr, bf, L.dinv32, nullptr,
                                       h->opt.omega, yf, nullptr, nullptr, nullptr));
          else
            PASE_TRY(launch_csr<double>(h, CSR_JACOBI, m, L.A, L.A.val, nullptr, x, nullptr, b, L.dinv, nullptr,
                                        h->opt.omega, y, nullptr, nullptr, nullptr));
        }
      }
      PASE_CUDA(cudaEventRecord(e1, h->stream));
      PASE_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      PASE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (h->opt.verbose >= 2)
        fprintf(stderr, "[pase]   level %d candidate: %s bs %d psm %d items %d cw %d: %.4f ms\n", l,
                cd.use ? "structured" : "CSR", cd.bs, cd.psm, cd.items, cd.cw, ms);
      if (ms < best) {
        best = ms;
        best_bs = cd.bs;
        best_use = cd.use;
        best_psm = cd.psm;
        best_items = cd.items;
        best_cw = cd.cw;
      }
    }
    L.A.block = best_bs;
    L.A.st_use = st ? best_use : 1;
    L.A.st_per_sm = best_psm;
    L.A.st_items = best_items;
    L.A.st_cw = best_cw;
    if (h->opt.verbose)
      fprintf(stderr, "[pase] autotune level %d: %s, %d threads/block, %d CTAs/SM, %d items, %d columns/thread "
              "(%.3f ms for 3 sweeps)\n", l, best_use ? "structured" : "CSR", best_bs, best_psm, best_items, best_cw, best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tuned_m = m;
  return tune_sygv(h);
}

// ------------------------------------------------------------------ workspace
static int reserve(pase_ctx* h, int m) {
  if (!h->ready) return fail(PASE_ERR_STATE, "pase_setup has not completed");
  if (m <= 0 || m % 8 != 0 || m > 256) return fail(PASE_ERR_INVALID_ARG, "block width m must be a positive multiple of 8, <= 256");
  if (h->w.m == m) return PASE_OK;
  if (h->w.m != 0) return fail(PASE_ERR_STATE, "a handle serves one block width; create another handle for a different m");
  Work& w = h->w;
  w.m = m;
  w.N = h->N;
  const int64_t N = h->N, NH = h->NH;
  const size_t nm = (size_t)N * m;
  PASE_TRY(dev_alloc_t(h, &w.R, nm));
  PASE_TRY(dev_alloc_t(h, &w.E, nm));
  PASE_TRY(dev_alloc_t(h, &w.T1, nm));
  PASE_TRY(dev_alloc_t(h, &w.T2, nm));
  PASE_TRY(dev_alloc_t(h, &w.W, nm));
  PASE_TRY(dev_alloc_t(h, &w.U, nm));
  PASE_TRY(dev_alloc_t(h, &w.lam, m));
  w.lb.assign(h->L, nullptr);
  w.lx.assign(h->L, nullptr);
  w.lt1.assign(h->L, nullptr);
  w.lt2.assign(h->L, nullptr);
  for (int l = 1; l < h->L; ++l) {
    const size_t k = (size_t)h->lv[l].A.nrows * m;
    PASE_TRY(dev_alloc_t(h, &w.lb[l], k));
    PASE_TRY(dev_alloc_t(h, &w.lx[l], k));
    PASE_TRY(dev_alloc_t(h, &w.lt1[l], k));
    PASE_TRY(dev_alloc_t(h, &w.lt2[l], k));
  }
  if (h->opt.precision == PASE_PREC_MIXED) {
    w.fb.assign(h->L, nullptr);
    w.fx.assign(h->L, nullptr);
    w.ft1.assign(h->L, nullptr);
    w.ft2.assign(h->L, nullptr);
    for (int l = 0; l < h->L; ++l) {
      const size_t k = (size_t)h->lv[l].A.nrows * m;
      PASE_TRY(dev_alloc_t(h, &w.fb[l], k));
      PASE_TRY(dev_alloc_t(h, &w.fx[l], k));
      PASE_TRY(dev_alloc_t(h, &w.ft1[l], k));
      PASE_TRY(dev_alloc_t(h, &w.ft2[l], k));
    }
  }
  if (h->opt.linear_solver == PASE_SOLVER_CG || h->opt.linear_solver == PASE_SOLVER_MGCG) {
    PASE_TRY(dev_alloc_t(h, &w.cgP, nm));
    PASE_TRY(dev_alloc_t(h, &w.cgQ, nm));
    PASE_TRY(dev_alloc_t(h, &w.cgs, 4 * (size_t)m));
  }
  const int64_t m3 = 3 * (int64_t)m;
  int64_t pd = std::max<int64_t>((int64_t)kReduceBlocksHost * 2 * m, std::min<int64_t>(608 * m3 * m3, 32ll << 20));
  pd = std::max<int64_t>(pd, m3 * m3 * 4);
  w.partial_bytes = pd * sizeof(double);
  PASE_TRY(dev_alloc(h, (void**)&w.partial, w.partial_bytes));
  PASE_TRY(dev_alloc_t(h, &w.norms, 4 * m));
  PASE_TRY(dev_alloc_t(h, &w.relres, m));
  PASE_TRY(dev_alloc_t(h, &w.aH, (size_t)NH * m));
  PASE_TRY(dev_alloc_t(h, &w.bH, (size_t)NH * m));
  PASE_TRY(dev_alloc_t(h, &w.GA, (size_t)m * m));
  PASE_TRY(dev_alloc_t(h, &w.GM, (size_t)m * m));
  PASE_TRY(dev_alloc_t(h, &w.CH, (size_t)NH * m));
  PASE_TRY(dev_alloc_t(h, &w.CW, (size_t)m * m));
  const size_t nc = (size_t)(NH + m);
  PASE_TRY(dev_alloc_t(h, &w.S, nc * m3));
  PASE_TRY(dev_alloc_t(h, &w.AS, nc * m3));
  PASE_TRY(dev_alloc_t(h, &w.BS, nc * m3));
  PASE_TRY(dev_alloc_t(h, &w.Xn, nc * m));
  PASE_TRY(dev_alloc_t(h, &w.AXn, nc * m));
  PASE_TRY(dev_alloc_t(h, &w.BXn, nc * m));
  PASE_TRY(dev_alloc_t(h, &w.Pn, nc * m));
  PASE_TRY(dev_alloc_t(h, &w.APn, nc * m));
  PASE_TRY(dev_alloc_t(h, &w.BPn, nc * m));
  PASE_TRY(dev_alloc_t(h, &w.Gq, (size_t)m3 * m3));
  PASE_TRY(dev_alloc_t(h, &w.Gb, (size_t)m3 * m3));
  PASE_TRY(dev_alloc_t(h, &w.Cs, (size_t)m3 * m));
  PASE_TRY(dev_alloc_t(h, &w.Rn, nc * m));
  PASE_TRY(dev_alloc_t(h, &w.coef, (size_t)m * m));
  PASE_TRY(dev_alloc_t(h, &w.ahat, (size_t)NH * m));
  PASE_TRY(dev_alloc_t(h, &w.schur, (size_t)m * m));
  w.eigwork_doubles = small_sygv_work_doubles((int)m3, m) + 64;
  PASE_TRY(dev_alloc_t(h, &w.eigwork, w.eigwork_doubles));
  PASE_TRY(dev_alloc_t(h, &w.smallvec, (size_t)16 * m));
  PASE_TRY(dev_alloc_t(h, &w.status, 8));
  PASE_TRY(dev_alloc_t(h, &w.colexp, 3 * 128));
  if (h->opt.spmm_df64) {
    PASE_TRY(dev_alloc_t(h, &w.dfh, nm));
    PASE_TRY(dev_alloc_t(h, &w.dfl, nm));
    PASE_TRY(dev_alloc_t(h, &w.df_flag, 1));
    PASE_CUDA(cudaMemsetAsync(w.df_flag, 0, sizeof(int), h->stream));
  }
  if (h->opt.aug_transform != PASE_AUG_PLAIN) {
    const size_t hm = (size_t)NH * m;
    PASE_TRY(dev_alloc_t(h, &w.Zt, hm));
    PASE_TRY(dev_alloc_t(h, &w.aT, hm));
    PASE_TRY(dev_alloc_t(h, &w.bT, hm));
    PASE_TRY(dev_alloc_t(h, &w.GAT, (size_t)m * m));
    PASE_TRY(dev_alloc_t(h, &w.GMT, (size_t)m * m));
    PASE_TRY(dev_alloc_t(h, &w.tr, hm));
    PASE_TRY(dev_alloc_t(h, &w.tz, hm));
    PASE_TRY(dev_alloc_t(h, &w.tp, hm));
    PASE_TRY(dev_alloc_t(h, &w.tq, hm));
    PASE_TRY(dev_alloc_t(h, &w.tsc, 4 * (size_t)m));
  }
  PASE_TRY(dev_alloc_t(h, &h->tc_err, 1));
  PASE_CUDA(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
  // Spaces no wider than the block eigensolver's [X, W, P] basis (3m columns) are solved
  // densely: the coarse pencil of the coarse start when N_H <= 3m, the augmented pencil of
  // step (c) when N_H + m <= 3m.
  if (NH <= m3) {
    w.coarse_dense = true;
    PASE_TRY(dev_alloc_t(h, &w.AHd, (size_t)NH * NH));
    PASE_TRY(dev_alloc_t(h, &w.MHd, (size_t)NH * NH));
    PASE_TRY(launch_csr_to_dense(h, NH, NH, h->AH.rowptr, h->AH.col, h->AH.val, w.AHd, NH));
    PASE_TRY(launch_csr_to_dense(h, NH, NH, h->AH.rowptr, h->AH.col, h->MH_val, w.MHd, NH));
  }
  if (NH + m <= m3) {
    const int64_t n = NH + m;
    w.aug_dense = true;
    PASE_TRY(dev_alloc_t(h, &w.Ad, (size_t)n * n));
    PASE_TRY(dev_alloc_t(h, &w.Bd, (size_t)n * n));
    PASE_TRY(dev_alloc_t(h, &w.Cd, (size_t)n * m));
  }
  PASE_TRY(dev_alloc_t(h, &w.ci, kCtlInts));
  PASE_TRY(dev_alloc_t(h, &w.cd, CD_COUNT));
  PASE_CUDA(cudaMemsetAsync(w.ci, 0, sizeof(int) * kCtlInts, h->stream));
  PASE_CUDA(cudaMemsetAsync(w.cd, 0, sizeof(double) * CD_COUNT, h->stream));
  PASE_CUDA(cudaMallocHost(&w.h_small, sizeof(double) * 16 * m));
  PASE_CUDA(cudaMallocHost(&w.h_status, sizeof(int) * 8));
  PASE_CUDA(cudaMallocHost(&w.h_ci, sizeof(int) * kCtlInts));
  PASE_CUDA(cudaMallocHost(&w.h_cd, sizeof(double) * CD_COUNT));
  if (h->opt.autotune) PASE_TRY(autotune(h));
  return PASE_OK;
}

// ------------------------------------------------------------------ multigrid
// One V-cycle for A_l x = b on level l (Alg. 1's linear solve): nu1 damped-Jacobi sweeps,
// residual, restriction P^T, recursion, prolongation P, nu2 sweeps; dense solve on the
// coarsest level.  x_zero: start from x = 0.  Level-l temporaries t1, t2 are used.
template <typename T>
struct LevelBufs {
  std::vector<T*> b, x, t1, t2;
};

template <typename T>
static const T* aval(const DevCSR& A);
template <>
const double* aval<double>(const DevCSR& A) {
  return A.val;
}
template <>
const float* aval<float>(const DevCSR& A) {
  return A.val32;
}
template <typename T>
static const T* dinv_of(const Level& L);
template <>
const double* dinv_of<double>(const Level& L) {
  return L.dinv;
}
template <>
const float* dinv_of<float>(const Level& L) {
  return L.dinv32;
}
template <typename T>
static const T* cinv_of(pase_ctx* h);
template <>
const double* cinv_of<double>(pase_ctx* h) {
  return h->cinv;
}
template <>
const float* cinv_of<float>(pase_ctx* h) {
  return h->cinv32;
}

// damped Jacobi sweeps from x (or from zero), result in `dst` (x or tmp), returns where
template <typename T>
static int jacobi_sweeps(pase_ctx* h, const Level& L, int m, const T* b, T* x, T* tmp, int sweeps,
                         bool x_zero, T** result) {
  const double om = h->opt.omega;
  T* cur = x;
  T* other = tmp;
  int s = 0;
  if (x_zero) {
    if (sweeps == 0) {
      PASE_TRY(launch_fill(h, 0, 0.0, nullptr));
      *result = nullptr;  // caller handles zero
      return PASE_OK;
    }
    // choose the first target so that the last sweep lands in x
    T* first = (sweeps % 2 == 1) ? x : tmp;
    PASE_TRY(launch_scale_dinv<T>(h, L.A.nrows, m, dinv_of<T>(L), om, b, first));
    cur = first;
    other = (first == x) ? tmp : x;
    s = 1;
  }
  for (; s < sweeps; ++s) {
    PASE_TRY(launch_csr<T>(h, CSR_JACOBI, m, L.A, aval<T>(L.A), nullptr, cur, nullptr, b, dinv_of<T>(L),
                           nullptr, om, other, nullptr, nullptr, nullptr));
    std::swap(cur, other);
  }
  *result = cur;
  return PASE_OK;
}

template <typename T>
static int vcycle(pase_ctx* h, LevelBufs<T>& B, int l, int m, bool x_zero);

// Fine level of the V-cycle with the learned smoother: each of the nu1 pre- and nu2
// post-smoothing sweeps is x <- x + S(b - A x) (the first from zero is x = S(b)).
template <typename T>
static int vcycle_fine_learned(pase_ctx* h, LevelBufs<T>& B, int m, bool x_zero) {
  const Level& L = h->lv[0];
  T* b = B.b[0];
  T* x = B.x[0];
  T* r = B.t1[0];
  const T* dinv = dinv_of<T>(L);
  for (int s = 0; s < h->opt.nu1; ++s) {
    if (x_zero && s == 0) {
      PASE_TRY(sm_apply<T>(h, m, b, m, dinv, x, m, false));
      continue;
    }
    PASE_TRY(launch_csr<T>(h, CSR_RESID, m, L.A, aval<T>(L.A), nullptr, x, nullptr, b, nullptr, nullptr, 0.0, r,
                           nullptr, nullptr, nullptr));
    PASE_TRY(sm_apply<T>(h, m, r, m, dinv, x, m, true));
  }
  if (x_zero && h->opt.nu1 == 0) PASE_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * L.A.nrows * m, h->stream));
  PASE_TRY(launch_csr<T>(h, CSR_RESID, m, L.A, aval<T>(L.A), nullptr, x, nullptr, b, nullptr, nullptr, 0.0, B.t2[0],
                         nullptr, nullptr, nullptr));
  PASE_TRY(launch_csr<T>(h, CSR_MV, m, L.PT, aval<T>(L.PT), nullptr, B.t2[0], nullptr, nullptr, nullptr, nullptr, 0.0,
                         B.b[1], nullptr, nullptr, nullptr));
  PASE_TRY(vcycle<T>(h, B, 1, m, true));
  PASE_TRY(launch_csr<T>(h, CSR_ADD, m, L.P, aval<T>(L.P), nullptr, B.x[1], nullptr, x, nullptr, nullptr, 0.0, x,
                         nullptr, nullptr, nullptr));
  for (int s = 0; s < h->opt.nu2; ++s) {
    PASE_TRY(launch_csr<T>(h, CSR_RESID, m, L.A, aval<T>(L.A), nullptr, x, nullptr, b, nullptr, nullptr, 0.0, r,
                           nullptr, nullptr, nullptr));
    PASE_TRY(sm_apply<T>(h, m, r, m, dinv, x, m, true));
  }
  return PASE_OK;
}

template <typename T>
static int vcycle(pase_ctx* h, LevelBufs<T>& B, int l, int m, bool x_zero) {
  const int Lc = h->L - 1;
  T* b = B.b[l];
  T* x = B.x[l];
  if (l == Lc) {
    return dense_mm<T>(h, h->ncoarsest, m, cinv_of<T>(h), b, x);
  }
  if (l == 0 && sm_active(h)) return vcycle_fine_learned<T>(h, B, m, x_zero);
  const Level& L = h->lv[l];
  T* cur = nullptr;
  PASE_TRY(jacobi_sweeps<T>(h, L, m, b, x, B.t1[l], h->opt.nu1, x_zero, &cur));
  if (cur == nullptr) {  // nu1 == 0 from zero
    PASE_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * L.A.nrows * m, h->stream));
    cur = x;
  }
  // residual r = b - A cur  -> t2 ; restrict b_{l+1} = P^T r
  PASE_TRY(launch_csr<T>(h, CSR_RESID, m, L.A, aval<T>(L.A), nullptr, cur, nullptr, b, nullptr, nullptr,
                         0.0, B.t2[l], nullptr, nullptr, nullptr));
  PASE_TRY(launch_csr<T>(h, CSR_MV, m, L.PT, aval<T>(L.PT), nullptr, B.t2[l], nullptr, nullptr, nullptr,
                         nullptr, 0.0, B.b[l + 1], nullptr, nullptr, nullptr));
  PASE_TRY(vcycle<T>(h, B, l + 1, m, true));
  // cur += P x_{l+1}
  PASE_TRY(launch_csr<T>(h, CSR_ADD, m, L.P, aval<T>(L.P), nullptr, B.x[l + 1], nullptr, cur, nullptr,
                         nullptr, 0.0, cur, nullptr, nullptr, nullptr));
  T* tmp = (cur == x) ? B.t1[l] : x;
  T* res = nullptr;
  // post-smoothing must end in x
  if (h->opt.nu2 > 0) {
    T* a = cur;
    T* o = tmp;
    for (int s = 0; s < h->opt.nu2; ++s) {
      PASE_TRY(launch_csr<T>(h, CSR_JACOBI, m, L.A, aval<T>(L.A), nullptr, a, nullptr, b, dinv_of<T>(L),
                             nullptr, h->opt.omega, o, nullptr, nullptr, nullptr));
      std::swap(a, o);
    }
    res = a;
  } else {
    res = cur;
  }
  if (res != x) PASE_CUDA(cudaMemcpyAsync(x, res, sizeof(T) * L.A.nrows * m, cudaMemcpyDeviceToDevice, h->stream));
  return PASE_OK;
}

static LevelBufs<double> fp64_bufs(pase_ctx* h) {
  LevelBufs<double> B;
  Work& w = h->w;
  B.b = w.lb;
  B.x = w.lx;
  B.t1 = w.lt1;
  B.t2 = w.lt2;
  B.b[0] = w.R;
  B.x[0] = w.E;
  B.t1[0] = w.T1;
  B.t2[0] = w.T2;
  return B;
}
static LevelBufs<float> fp32_bufs(pase_ctx* h) {
  LevelBufs<float> B;
  Work& w = h->w;
  B.b = w.fb;
  B.x = w.fx;
  B.t1 = w.ft1;
  B.t2 = w.ft2;
  return B;
}

// Z = B R with B one V-cycle from zero (R in w.R, Z in w.E); FP32 inside in MIXED precision.
static int vcycle_precond(pase_ctx* h) {
  Work& w = h->w;
  const size_t nm = (size_t)h->N * w.m;
  if (h->opt.precision == PASE_PREC_MIXED) {
    LevelBufs<float> B = fp32_bufs(h);
    PASE_TRY(launch_f64_to_f32(h, nm, w.R, B.b[0]));
    PASE_TRY(vcycle<float>(h, B, 0, w.m, true));
    return launch_f32_to_f64(h, nm, B.x[0], w.E);
  }
  LevelBufs<double> B = fp64_bufs(h);
  return vcycle<double>(h, B, 0, w.m, true);
}

// Step (a), CG forms: s (preconditioned) CG steps per column on A w = M u lambda from
// w = u.  The initial residual is R = M U Lambda - A U, already in w.R.  All scalars stay
// on the device (column inner products, ratios), so the step has no host round trip.
// Buffers: X = W, R = w.R, Z = w.E (MGCG) or R itself (CG), P = w.cgP, Q = A P = w.cgQ.
static int step_cg(pase_ctx* h, const double* U, double* W) {
  Work& w = h->w;
  const int m = w.m;
  const int64_t N = h->N;
  const int s = std::max(1, h->opt.inner_steps);
  const bool pre = h->opt.linear_solver == PASE_SOLVER_MGCG;
  const DevCSR& A = h->lv[0].A;
  double* rz = w.cgs;
  double* rz_new = w.cgs + m;
  double* pq = w.cgs + 2 * m;
  double* coef = w.cgs + 3 * m;
  double* Z = pre ? w.E : w.R;
  if (W != U) PASE_CUDA(cudaMemcpyAsync(W, U, sizeof(double) * N * m, cudaMemcpyDeviceToDevice, h->stream));
  if (pre) PASE_TRY(vcycle_precond(h));
  PASE_TRY(launch_coldot(h, N, m, w.R, Z, rz));
  PASE_CUDA(cudaMemcpyAsync(w.cgP, Z, sizeof(double) * N * m, cudaMemcpyDeviceToDevice, h->stream));
  int nb = 0;
  for (int k = 0; k < s; ++k) {
    // Q = A P with the column sums of P .* Q in the same pass
    PASE_TRY(launch_csr<double>(h, CSR_MVDOT, m, A, A.val, nullptr, w.cgP, nullptr, nullptr, nullptr, nullptr,
                                0.0, w.cgQ, nullptr, w.partial, &nb));
    PASE_TRY(launch_reduce_partials(h, nb, m, w.partial, pq));
    PASE_TRY(launch_ratio(h, m, rz, pq, coef));  // alpha
    PASE_TRY(launch_cg_update(h, N, m, coef, w.cgP, w.cgQ, W, w.R));
    if (k + 1 == s) break;
    if (pre) PASE_TRY(vcycle_precond(h));
    PASE_TRY(launch_coldot(h, N, m, w.R, Z, rz_new));
    PASE_TRY(launch_ratio(h, m, rz_new, rz, coef));  // beta
    PASE_TRY(launch_cg_dir(h, N, m, coef, Z, w.cgP));
    std::swap(rz, rz_new);
  }
  return PASE_OK;
}

// Step (a): W = U + E, E from s V-cycles on A E = R (R already in w.R), or the CG forms.
static int step_linear_solve(pase_ctx* h, const double* U, double* W) {
  Work& w = h->w;
  const int m = w.m;
  const int s = std::max(1, h->opt.inner_steps);
  const size_t nm = (size_t)h->N * m;
  if (h->opt.linear_solver == PASE_SOLVER_CG || h->opt.linear_solver == PASE_SOLVER_MGCG) return step_cg(h, U, W);
  if (h->opt.linear_solver != PASE_SOLVER_VCYCLE) return fail(PASE_ERR_INVALID_ARG, "unknown linear solver");
  if (h->opt.precision == PASE_PREC_MIXED) {
    LevelBufs<float> B = fp32_bufs(h);
    PASE_TRY(launch_f64_to_f32(h, nm, w.R, B.b[0]));
    for (int c = 0; c < s; ++c) PASE_TRY(vcycle<float>(h, B, 0, m, c == 0));
    PASE_TRY(launch_add_f32_to_f64(h, nm, U, B.x[0], W));
  } else {
    LevelBufs<double> B = fp64_bufs(h);
    for (int c = 0; c < s; ++c) PASE_TRY(vcycle<double>(h, B, 0, m, c == 0));
    PASE_TRY(launch_axpy(h, nm, 1.0, w.E, U, W));
  }
  return PASE_OK;
}

// Step (a) through a CUDA graph.  The graph bakes in the addresses of U and W, so it is
// captured only once the same (U, W) pair has been seen on two calls in a row (the first
// of them runs eagerly and also sets up kernel attributes); later calls with that pair
// replay it, calls with other buffers run eagerly.
static int step_linear_solve_graphed(pase_ctx* h, const double* U, double* W) {
  if (!h->opt.use_graphs || !h->graphs_ok || h->stream == nullptr || h->prof_kernel >= 0)
    return step_linear_solve(h, U, W);
  if (h->ls_graph && h->ls_graph_U == U && h->ls_graph_W == W) {
    PASE_CUDA(cudaGraphLaunch(h->ls_graph, h->stream));
    h->launches += h->ls_graph_kernels;
    h->replayed += h->ls_graph_kernels;
    h->graph_launches++;
    return PASE_OK;
  }
  const bool stable = (h->ls_last_U == U && h->ls_last_W == W);
  h->ls_last_U = U;
  h->ls_last_W = W;
  if (!stable) return step_linear_solve(h, U, W);
  if (h->ls_graph) {
    cudaGraphExecDestroy(h->ls_graph);
    h->ls_graph = nullptr;
  }
  const int64_t l0 = h->launches;
  PASE_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = step_linear_solve(h, U, W);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  const int64_t captured = h->launches - l0;
  h->launches = l0;
  if (rc != PASE_OK || e != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    h->graphs_ok = false;  // fall back to eager launches for this handle
    return step_linear_solve(h, U, W);
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    h->graphs_ok = false;
    return step_linear_solve(h, U, W);
  }
  h->ls_graph = ex;
  h->ls_graph_U = U;
  h->ls_graph_W = W;
  h->ls_graph_kernels = captured;
  PASE_CUDA(cudaGraphLaunch(ex, h->stream));
  h->launches += captured;
  h->replayed += captured;
  h->graph_launches++;
  return PASE_OK;
}

// Residual R = M U Lambda - A U and relative residuals into w.relres (device).
// The fused fine-level products A_h X, M_h X (and the eigen-residual) in double-float
// arithmetic when the handle has the split values (spmm_df64), else in FP64.
static bool use_df64(const pase_ctx* h) { return h->opt.spmm_df64 && h->A0h && h->w.dfh; }
static int fine_products(pase_ctx* h, int mode, const double* X, const double* lam, double* Y1, double* Y2,
                         int* nb) {
  Work& w = h->w;
  const int m = w.m;
  if (use_df64(h)) {
    PASE_TRY(launch_split_df64(h, h->N * m, X, w.dfh, w.dfl, w.df_flag));
    return launch_csr_df64(h, mode, m, h->lv[0].A, h->A0h, h->A0l, h->M0h, h->M0l, w.dfh, w.dfl, lam, Y1, Y2,
                           w.partial, nb);
  }
  return launch_csr<double>(h, mode, m, h->lv[0].A, h->lv[0].A.val, h->M0_val, X, nullptr, nullptr, nullptr, lam,
                            0.0, Y1, Y2, w.partial, nb);
}

// PASE_ERR_NAN if a double-float split met a value outside 2^+-100 (clears the flag)
static int df_check(pase_ctx* h) {
  if (!h->w.df_flag) return PASE_OK;
  int f = 0;
  PASE_CUDA(cudaMemcpyAsync(&f, h->w.df_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PASE_CUDA(cudaStreamSynchronize(h->stream));
  if (f) {
    PASE_CUDA(cudaMemsetAsync(h->w.df_flag, 0, sizeof(int), h->stream));
    return fail(PASE_ERR_NAN, "a block entry above 2^100 (or not finite) met the double-float products; "
                              "set spmm_df64 = 0 for such data");
  }
  return PASE_OK;
}

static int step_residual(pase_ctx* h, const double* U, const double* lam, double* R) {
  Work& w = h->w;
  const int m = w.m;
  int nb = 0;
  PASE_TRY(fine_products(h, CSR_EIGRES, U, lam, R, nullptr, &nb));
  PASE_TRY(launch_reduce_partials(h, nb, 2 * m, w.partial, w.norms));
  PASE_TRY(launch_relres(h, m, w.norms, lam, w.relres));
  return PASE_OK;
}

// Step (b): aH = P^T A W, bH = P^T M W, GA = W^T A W, GM = W^T M W.
static int step_project(pase_ctx* h, const double* W, double* aH, double* bH, double* GA, double* GM) {
  Work& w = h->w;
  const int m = w.m;
  PASE_TRY(fine_products(h, CSR_MV_AM, W, nullptr, w.T1, w.T2, nullptr));
  PASE_TRY(launch_csr<double>(h, CSR_MV2, m, h->PdT, h->PdT.val, nullptr, w.T1, w.T2, nullptr, nullptr,
                              nullptr, 0.0, aH, bH, nullptr, nullptr));
  if (h->opt.split_gemm && ts_gram2_split_ok(h->N, m, h->num_sms, w))
    return ts_gram2_split(h, h->N, m, W, w.T1, w.T2, GA, GM, m, w.colexp, h->tc_err);
  PASE_TRY(ts_gram(h, h->N, m, m, W, m, w.T1, m, GA, m, true));
  PASE_TRY(ts_gram(h, h->N, m, m, W, m, w.T2, m, GM, m, true));
  return PASE_OK;
}

// Step (d): U = W C_W + P C_H.
static int step_prolongate(pase_ctx* h, const double* W, const double* CH, const double* CW, double* U) {
  const int m = h->w.m;
  if (h->opt.split_gemm && ts_gemm_split_ok(m, m, W, m, U, m))
    PASE_TRY(ts_gemm_split(h, h->N, m, m, W, m, CW, m, U, m, h->tc_err));
  else
    PASE_TRY(ts_gemm(h, h->N, m, m, 1.0, W, m, CW, m, 0.0, U, m));
  PASE_TRY(launch_csr<double>(h, CSR_ADD, m, h->Pd, h->Pd.val, nullptr, CH, nullptr, U, nullptr, nullptr, 0.0,
                              U, nullptr, nullptr, nullptr));
  return PASE_OK;
}

// Read (and clear) the flag of a tensor-core wait that ran out of its limit.
static int tc_check(pase_ctx* h) {
  if (!h->tc_err) return PASE_OK;
  PASE_CUDA(cudaMemcpyAsync(h->w.h_status + 7, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PASE_CUDA(cudaStreamSynchronize(h->stream));
  if (h->w.h_status[7]) {
    PASE_CUDA(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->stream));
    return fail(PASE_ERR_TIMEOUT, "a tensor-core or bulk-copy wait (split GEMM, stencil kernel) ran out of its limit");
  }
  return PASE_OK;
}

// ------------------------------------------------------------------ step (c)
// The augmented pencil acts on blocks Y [n_c][ld] (rows 0..N_H-1: coarse coefficients,
// rows N_H..N_H+m-1: coefficients of W), k columns:
//   A^ Y = [A_H Y1 + aH Y2 ; aH^T Y1 + GA Y2],  B^ Y = [M_H Y1 + bH Y2 ; bH^T Y1 + GM Y2]
// (the block product of §4, computed without forming the dense pencil).
static int aug_apply(pase_ctx* h, int k, const double* Y, int ld, double* AY, double* BY, int ldo,
                     const double* aH, const double* bH, const double* GA, const double* GM) {
  const int m = h->w.m;
  const int64_t NH = h->NH;
  if (k % 8 != 0) return fail(PASE_ERR_INVALID_ARG, "aug_apply: k must be a multiple of 8");
  PASE_TRY(launch_csr<double>(h, CSR_MV_AM, k, h->AH, h->AH.val, h->MH_val, Y, nullptr, nullptr, nullptr,
                              nullptr, 0.0, AY, BY, nullptr, nullptr, ld, ldo));
  const double* Y2 = Y + NH * ld;
  PASE_TRY(ts_gemm(h, NH, m, k, 1.0, aH, m, Y2, ld, 1.0, AY, ldo));
  PASE_TRY(ts_gemm(h, NH, m, k, 1.0, bH, m, Y2, ld, 1.0, BY, ldo));
  PASE_TRY(ts_gram(h, NH, m, k, aH, m, Y, ld, AY + NH * ldo, ldo, false));
  PASE_TRY(ts_gram(h, NH, m, k, bH, m, Y, ld, BY + NH * ldo, ldo, false));
  PASE_TRY(small_gemm(h, m, k, m, 1.0, GA, m, false, Y2, ld, 1.0, AY + NH * ldo, ldo));
  PASE_TRY(small_gemm(h, m, k, m, 1.0, GM, m, false, Y2, ld, 1.0, BY + NH * ldo, ldo));
  return PASE_OK;
}

// A_H^-1 approximated by a V-cycle from the coarse level (exact when V_H is the coarsest
// multigrid level): y = Ainv(r) for r [N_H][ld] (first m columns) -> y [N_H][ldo].
static int coarse_apply(pase_ctx* h, const double* r, int ld, double* y, int ldo) {
  const int m = h->w.m;
  const int c = h->coarse_level;
  LevelBufs<double> B = fp64_bufs(h);
  PASE_TRY(launch_copy_cols(h, h->NH, m, r, ld, B.b[c], m));
  PASE_TRY(vcycle<double>(h, B, c, m, true));
  PASE_TRY(launch_copy_cols(h, h->NH, m, B.x[c], m, y, ldo));
  return PASE_OK;
}


// Preconditioner T ~ A^^-1 from the block factorisation behind PRECOND-A (§4, Alg. 5
// step 1): with ahat = Ainv aH and S = GA - aH^T ahat (PRECOND-A's alpha~),
//   y1' = Ainv r1,  y2 = S^-1 (r2 - aH^T y1'),  y1 = y1' - ahat y2.
// Ainv is the coarse V-cycle, so T is symmetric positive definite.
// blockdiag: the block-diagonal preconditioner [Ainv r1; GA^-1 r2] (no coupling terms).
static int aug_precond(pase_ctx* h, const double* R, int ld, double* Y, int ldo, const double* aH,
                       bool blockdiag = false) {
  Work& w = h->w;
  const int m = w.m;
  const int64_t NH = h->NH;
  PASE_TRY(coarse_apply(h, R, ld, Y, ldo));
  double* y2 = Y + NH * ldo;
  if (blockdiag) {
    PASE_TRY(launch_copy_cols(h, m, m, R + NH * ld, ld, y2, ldo));
    return small_chol_solve(h, m, m, w.schur, m, y2, ldo, w.status + 2, false);
  }
  PASE_TRY(ts_gram(h, NH, m, m, aH, m, Y, ldo, w.coef, m, false));
  PASE_TRY(launch_geam(h, m, m, 1.0, R + NH * ld, ld, -1.0, w.coef, m, y2, ldo));
  PASE_TRY(small_chol_solve(h, m, m, w.schur, m, y2, ldo, w.status + 2, false));
  PASE_TRY(ts_gemm(h, NH, m, m, -1.0, w.ahat, m, y2, ldo, 1.0, Y, ldo));
  return PASE_OK;
}

static int aug_precond_setup(pase_ctx* h, const double* aH, const double* GA, bool blockdiag = false) {
  Work& w = h->w;
  const int m = w.m;
  if (blockdiag) {  // S = GA
    PASE_TRY(launch_copy_cols(h, m, m, GA, m, w.schur, m));
  } else {
    PASE_TRY(coarse_apply(h, aH, m, w.ahat, m));
    PASE_TRY(ts_gram(h, h->NH, m, m, aH, m, w.ahat, m, w.coef, m, false));
    PASE_TRY(launch_geam(h, m, m, 1.0, GA, m, -1.0, w.coef, m, w.schur, m));
  }
  // factor (the Cholesky reads the lower triangle only)
  PASE_TRY(small_chol_solve(h, m, 0, w.schur, m, nullptr, 0, w.status + 1, true));
  return PASE_OK;
}

// Z ~ M_H^-1 B for B [N_H][m]: `steps` Jacobi-preconditioned CG steps per column from
// zero on the coarse mass matrix (well conditioned: a dozen steps gain about two digits).
static int coarse_mass_solve(pase_ctx* h, const double* B, double* Z, int steps) {
  Work& w = h->w;
  const int m = w.m;
  const int64_t NH = h->NH;
  DevCSR Mc = h->AH;
  Mc.val = h->MH_val;
  double *r = w.tr, *z = w.tz, *p = w.tp, *q = w.tq;
  double *rz = w.tsc, *rz_new = w.tsc + m, *pq = w.tsc + 2 * m, *coef = w.tsc + 3 * m;
  const size_t bytes = sizeof(double) * NH * m;
  PASE_CUDA(cudaMemsetAsync(Z, 0, bytes, h->stream));
  PASE_CUDA(cudaMemcpyAsync(r, B, bytes, cudaMemcpyDeviceToDevice, h->stream));
  PASE_TRY(launch_scale_dinv<double>(h, NH, m, h->MH_dinv, 1.0, r, z));
  PASE_TRY(launch_coldot(h, NH, m, r, z, rz));
  PASE_CUDA(cudaMemcpyAsync(p, z, bytes, cudaMemcpyDeviceToDevice, h->stream));
  for (int k = 0; k < steps; ++k) {
    int nb = 0;
    PASE_TRY(launch_csr<double>(h, CSR_MVDOT, m, Mc, Mc.val, nullptr, p, nullptr, nullptr, nullptr, nullptr, 0.0, q,
                                nullptr, w.partial, &nb));
    PASE_TRY(launch_reduce_partials(h, nb, m, w.partial, pq));
    PASE_TRY(launch_ratio(h, m, rz, pq, coef));
    PASE_TRY(launch_cg_update(h, NH, m, coef, p, q, Z, r));
    if (k + 1 == steps) break;
    PASE_TRY(launch_scale_dinv<double>(h, NH, m, h->MH_dinv, 1.0, r, z));
    PASE_TRY(launch_coldot(h, NH, m, r, z, rz_new));
    PASE_TRY(launch_ratio(h, m, rz_new, rz, coef));
    PASE_TRY(launch_cg_dir(h, NH, m, coef, z, p));
    std::swap(rz, rz_new);
  }
  return PASE_OK;
}

// The congruence T = [[I, Z], [0, I]] of §4 applied to the augmented pencil: with
// D_A = A_H Z - aH and D_B = M_H Z - bH,
//   aT = -D_A,  GAT = GA + Z^T D_A - aH^T Z   (= GA - Z^T aH - aH^T Z + Z^T A_H Z)
//   bT = -D_B,  GMT = GM + Z^T D_B - bH^T Z
// so that [[A_H, aT],[aT^T, GAT]] = T^-T A_Hh T^-1 and likewise for B_Hh, for any Z.
static int aug_congruence(pase_ctx* h, const double* aH, const double* bH, const double* GA, const double* GM) {
  Work& w = h->w;
  const int m = w.m;
  const int64_t NH = h->NH;
  PASE_TRY(launch_csr<double>(h, CSR_MV_AM, m, h->AH, h->AH.val, h->MH_val, w.Zt, nullptr, nullptr, nullptr, nullptr,
                              0.0, w.tr, w.tz, nullptr, nullptr));
  PASE_TRY(launch_geam(h, NH, m, 1.0, w.tr, m, -1.0, aH, m, w.tr, m));  // D_A
  PASE_TRY(launch_geam(h, NH, m, 1.0, w.tz, m, -1.0, bH, m, w.tz, m));  // D_B
  PASE_TRY(launch_geam(h, NH, m, -1.0, w.tr, m, 0.0, w.tr, m, w.aT, m));
  PASE_TRY(launch_geam(h, NH, m, -1.0, w.tz, m, 0.0, w.tz, m, w.bT, m));
  PASE_TRY(ts_gram(h, NH, m, m, w.Zt, m, w.tr, m, w.coef, m, false));   // Z^T D_A
  PASE_TRY(launch_geam(h, m, m, 1.0, GA, m, 1.0, w.coef, m, w.GAT, m));
  PASE_TRY(ts_gram(h, NH, m, m, aH, m, w.Zt, m, w.coef, m, false));     // aH^T Z
  PASE_TRY(launch_geam(h, m, m, 1.0, w.GAT, m, -1.0, w.coef, m, w.GAT, m));
  PASE_TRY(ts_gram(h, NH, m, m, w.Zt, m, w.tz, m, w.coef, m, false));   // Z^T D_B
  PASE_TRY(launch_geam(h, m, m, 1.0, GM, m, 1.0, w.coef, m, w.GMT, m));
  PASE_TRY(ts_gram(h, NH, m, m, bH, m, w.Zt, m, w.coef, m, false));     // bH^T Z
  PASE_TRY(launch_geam(h, m, m, 1.0, w.GMT, m, -1.0, w.coef, m, w.GMT, m));
  return PASE_OK;
}

// Operators of the block eigensolver.
struct BlockOp {
  int64_t n;
  int kind;  // 0: augmented pencil, 1: coarse pencil (A_H, M_H)
  const double *aH, *bH, *GA, *GM;
  bool blockdiag = false;  // augmented pencil: block-diagonal preconditioner
};

static int op_apply(pase_ctx* h, const BlockOp& op, const double* Y, int ld, double* AY, double* BY, int ldo) {
  if (op.kind == 0) return aug_apply(h, h->w.m, Y, ld, AY, BY, ldo, op.aH, op.bH, op.GA, op.GM);
  return launch_csr<double>(h, CSR_MV_AM, h->w.m, h->AH, h->AH.val, h->MH_val, Y, nullptr, nullptr, nullptr,
                            nullptr, 0.0, AY, BY, nullptr, nullptr, ld, ldo);
}
static int op_precond(pase_ctx* h, const BlockOp& op, const double* R, int ld, double* Y, int ldo) {
  if (op.kind == 0) return aug_precond(h, R, ld, Y, ldo, op.aH, op.blockdiag);
  return coarse_apply(h, R, ld, Y, ldo);
}

static int sync_small(pase_ctx* h, const double* dsrc, int count, const int* dstatus, int nstatus) {
  Work& w = h->w;
  if (count) PASE_CUDA(cudaMemcpyAsync(w.h_small, dsrc, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
  if (nstatus) PASE_CUDA(cudaMemcpyAsync(w.h_status, dstatus, sizeof(int) * nstatus, cudaMemcpyDeviceToHost, h->stream));
  PASE_CUDA(cudaStreamSynchronize(h->stream));
  return PASE_OK;
}

// Block eigensolver for the m smallest pairs of (A, B): locally optimal block
// preconditioned iteration on the basis [X, W, P] (W = T R, P = previous step), each
// step a Rayleigh-Ritz on the basis (the X, P, W blocks and the Rayleigh-Ritz of GCG_AUG,
// Alg. 4; P is the last update direction).  W and P are B-orthogonalised against X twice
// and every operator product is recomputed (implicit updates lose accuracy once the
// block has converged past ~1e-9); converged columns are soft-locked.
// On entry S[:, 0:m] holds the start block; on exit S[:, 0:m] = X (B-orthonormal), lam
// (device) its Ritz values.
// Recorded into a CUDA graph: the first pass (no P block yet) is unrolled, the others run
// in a conditional WHILE node; each pass's test (k_ctl_inner_check: the first nconv
// columns at relative residual <= tol, where tol is *tol_dev or tol_fixed; stagnation;
// maxit passes) and the small eigensolve's status steer IF nodes, so no pass waits on
// the host.  Errors (NaN, a start block that is not B-independent) land in the control
// block.
static int eig_pass(pase_ctx* h, const BlockOp& op, double* lam, const double* tol_dev, double tol_fixed, int maxit,
                    int nconv, bool haveP) {
  Work& w = h->w;
  const int m = w.m;
  const int m3 = 3 * m;
  const int64_t n = op.n;
  double *S = w.S, *AS = w.AS, *BS = w.BS;
  int nb = 0;
  PASE_TRY(launch_block_resid(h, n, m, AS, BS, m3, lam, w.Rn, m, &nb));
  PASE_TRY(launch_reduce_partials(h, nb, 2 * m, w.partial, w.norms));
  PASE_TRY(launch_relres(h, m, w.norms, lam, w.smallvec));
  PASE_TRY(launch_ctl_inner_check(h, nconv, w.smallvec, tol_dev, tol_fixed, maxit));
  return cond_node(h, false, w.ci + CI_IN_GO, [&]() -> int {
    // soft locking: converged columns contribute no new search direction
    PASE_TRY(launch_zero_cols_if(h, n, m, m, w.smallvec, tol_fixed, w.Rn, tol_dev));
    // W = T R, B-orthogonal to X (two Gram-Schmidt passes), products computed afresh
    double* Wb = S + m;
    PASE_TRY(op_precond(h, op, w.Rn, m, Wb, m3));
    for (int pass = 0; pass < 2; ++pass) {
      PASE_TRY(ts_gram(h, n, m, m, BS, m3, Wb, m3, w.coef, m, false));
      PASE_TRY(ts_gemm(h, n, m, m, -1.0, S, m3, w.coef, m, 1.0, Wb, m3));
    }
    PASE_TRY(op_apply(h, op, Wb, m3, AS + m, BS + m, m3));
    int nbw = 2 * m;
    if (haveP) {
      double* Pb = S + 2 * m;
      PASE_TRY(launch_copy_cols(h, n, m, w.Pn, m, Pb, m3));
      for (int pass = 0; pass < 2; ++pass) {
        PASE_TRY(ts_gram(h, n, m, m, BS, m3, Pb, m3, w.coef, m, false));
        PASE_TRY(ts_gemm(h, n, m, m, -1.0, S, m3, w.coef, m, 1.0, Pb, m3));
      }
      PASE_TRY(op_apply(h, op, Pb, m3, AS + 2 * m, BS + 2 * m, m3));
      nbw = m3;
    }
    PASE_TRY(ts_gram(h, n, nbw, nbw, S, m3, AS, m3, w.Gq, m3, true));
    PASE_TRY(ts_gram(h, n, nbw, nbw, S, m3, BS, m3, w.Gb, m3, true));
    PASE_TRY(small_sygv(h, nbw, m, w.Gq, m3, w.Gb, m3, w.smallvec + m, w.Cs, m, w.status));
    PASE_TRY(launch_ctl_status(h, w.status, false));  // fewer than m independent directions: stop
    return cond_node(h, false, w.ci + CI_IN_OK, [&]() -> int {
      // X = S C, P = S[:, m:] C[m:, :]; products of X recomputed
      PASE_TRY(ts_gemm(h, n, nbw, m, 1.0, S, m3, w.Cs, m, 0.0, w.Xn, m));
      PASE_TRY(ts_gemm(h, n, nbw - m, m, 1.0, S + m, m3, w.Cs + (size_t)m * m, m, 0.0, w.Pn, m));
      PASE_TRY(launch_copy_cols(h, n, m, w.Xn, m, S, m3));
      PASE_TRY(op_apply(h, op, S, m3, AS, BS, m3));
      PASE_CUDA(cudaMemcpyAsync(lam, w.smallvec + m, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->stream));
      return PASE_OK;
    });
  });
}

static int block_eigensolver(pase_ctx* h, const BlockOp& op, double* lam, const double* tol_dev, double tol_fixed,
                             int maxit, int nconv) {
  Work& w = h->w;
  const int m = w.m;
  const int m3 = 3 * m;
  const int64_t n = op.n;
  double *S = w.S, *AS = w.AS, *BS = w.BS;
  if (nconv <= 0 || nconv > m) nconv = m;
  // initial Rayleigh-Ritz on the start block
  PASE_TRY(op_apply(h, op, S, m3, AS, BS, m3));
  PASE_TRY(ts_gram(h, n, m, m, S, m3, AS, m3, w.Gq, m3, true));
  PASE_TRY(ts_gram(h, n, m, m, S, m3, BS, m3, w.Gb, m3, true));
  PASE_TRY(small_sygv(h, m, m, w.Gq, m3, w.Gb, m3, lam, w.Cs, m, w.status));
  PASE_TRY(launch_ctl_status(h, w.status, true));  // start block not B-independent: error
  PASE_TRY(ts_gemm(h, n, m, m, 1.0, S, m3, w.Cs, m, 0.0, w.Xn, m));
  PASE_TRY(launch_copy_cols(h, n, m, w.Xn, m, S, m3));
  PASE_TRY(op_apply(h, op, S, m3, AS, BS, m3));
  PASE_TRY(launch_ctl_inner_init(h));
  PASE_TRY(eig_pass(h, op, lam, tol_dev, tol_fixed, maxit, nconv, false));
  return cond_node(
      h, true, w.ci + CI_IN_CONT, [&]() -> int { return eig_pass(h, op, lam, tol_dev, tol_fixed, maxit, nconv, true); },
      maxit + 1);
}

// Step (c) when the augmented space is no wider than the block eigensolver's basis
// (N_H + m <= 3m, small coarse spaces): the pencil is assembled densely and its m
// smallest pairs come from one generalized eigensolve (M-orthonormal, exact to rounding;
// the congruences of §4 leave the pairs unchanged, so they are not applied).
static int dense_step_c(pase_ctx* h, const double* aH, const double* bH, const double* GA, const double* GM,
                        double* lam, double* CH, double* CW) {
  Work& w = h->w;
  const int m = w.m;
  const int64_t NH = h->NH, n = NH + m;
  const double* src[2][3] = {{w.AHd, aH, GA}, {w.MHd, bH, GM}};
  double* dst[2] = {w.Ad, w.Bd};
  for (int q = 0; q < 2; ++q) {
    if (NH) PASE_TRY(launch_geam(h, NH, (int)NH, 1.0, src[q][0], NH, 0.0, src[q][0], NH, dst[q], n));
    PASE_TRY(launch_copy_cols(h, NH, m, src[q][1], m, dst[q] + NH, (int)n));
    PASE_TRY(launch_transpose(h, NH, m, src[q][1], m, dst[q] + NH * n, n));
    PASE_TRY(launch_copy_cols(h, m, m, src[q][2], m, dst[q] + NH * n + NH, (int)n));
  }
  PASE_TRY(small_sygv(h, (int)n, m, w.Ad, (int)n, w.Bd, (int)n, lam, w.Cd, m, w.status));
  PASE_TRY(launch_ctl_status(h, w.status, true));
  PASE_TRY(launch_ctl_put(h, w.ci + CI_AUG_IT, 1, true, nullptr, 0.0));
  PASE_TRY(launch_copy_cols(h, NH, m, w.Cd, m, CH, m));
  return launch_copy_cols(h, m, m, w.Cd + NH * m, m, CW, m);
}

// Step (c), recorded: the m smallest pairs of the augmented pencil, warm start u_H = 0,
// gamma = I, to the inner tolerance held in the control block.
static int record_step_c(pase_ctx* h, const double* aH, const double* bH, const double* GA, const double* GM,
                         double* lam, double* CH, double* CW) {
  Work& w = h->w;
  if (w.aug_dense) return dense_step_c(h, aH, bH, GA, GM, lam, CH, CW);
  const int m = w.m;
  const int m3 = 3 * m;
  const int64_t NH = h->NH, nc = NH + m;
  const int tr = h->opt.aug_transform;
  if (tr != PASE_AUG_PLAIN) {  // §4: the pencil seen through T = [[I, Z], [0, I]]
    if (tr == PASE_AUG_PRECOND_A) PASE_TRY(coarse_apply(h, aH, m, w.Zt, m));     // Z ~ A_H^-1 aH
    else PASE_TRY(coarse_mass_solve(h, bH, w.Zt, 12));                        // Z ~ M_H^-1 bH
    PASE_TRY(aug_congruence(h, aH, bH, GA, GM));
    aH = w.aT;
    bH = w.bT;
    GA = w.GAT;
    GM = w.GMT;
  }
  const bool blockdiag = tr == PASE_AUG_PRECOND_B;
  PASE_TRY(aug_precond_setup(h, aH, GA, blockdiag));
  // start block: the warm start u_H = 0, gamma = I, i.e. [0; I], which the congruence maps
  // to [Z; I]
  PASE_CUDA(cudaMemsetAsync(w.S, 0, sizeof(double) * nc * m3, h->stream));
  PASE_TRY(launch_set_identity_rows(h, NH, m, m3, w.S));
  if (tr != PASE_AUG_PLAIN) PASE_TRY(launch_copy_cols(h, NH, m, w.Zt, m, w.S, m3));
  BlockOp op{nc, 0, aH, bH, GA, GM, blockdiag};
  PASE_TRY(block_eigensolver(h, op, lam, w.cd + CD_AUG_TOL, 0.0, h->opt.aug_max_iter, h->aug_nconv));
  PASE_TRY(launch_copy_cols(h, NH, m, w.S, m3, CH, m));
  PASE_TRY(launch_copy_cols(h, m, m, w.S + NH * m3, m3, CW, m));
  if (tr != PASE_AUG_PLAIN)  // back to the original basis: u_H = u~_H - Z gamma~ (Alg. 5 step 3)
    PASE_TRY(ts_gemm(h, NH, m, m, -1.0, w.Zt, m, CW, m, 1.0, CH, m));
  return PASE_OK;
}

static uint64_t key_of(const void* p) { return (uint64_t)(uintptr_t)p; }
static uint64_t key_of(double v) {
  uint64_t u;
  memcpy(&u, &v, sizeof(u));
  return u;
}

// Step (c): recorded once per set of buffers and replayed (one graph launch); inside a
// recording it is recorded in place.
static int step_augmented_eig(pase_ctx* h, const double* aH, const double* bH, const double* GA,
                              const double* GM, double* lam, double* CH, double* CW) {
  auto rec = [=]() -> int { return record_step_c(h, aH, bH, GA, GM, lam, CH, CW); };
  if (recording(h)) return rec();
  const std::vector<uint64_t> key = {key_of(aH), key_of(bH), key_of(GA), key_of(GM), key_of(lam), key_of(CH),
                                     key_of(CW), (uint64_t)h->aug_nconv};
  if (!h->g_stepc.exec || h->g_stepc.key != key) {
    PASE_TRY(graph_record(h, h->g_stepc, rec));
    h->g_stepc.key = key;
  }
  return graph_launch(h, h->g_stepc);
}

// Alg. 3 steps 1-2: coarse eigenpairs of (A_H, M_H), interpolated: U = I_H^h u_H.
static int record_coarse_start(pase_ctx* h, double* U, double* lam) {
  Work& w = h->w;
  const int m = w.m;
  const int m3 = 3 * m;
  const int64_t NH = h->NH;
  if (w.coarse_dense) {  // a coarse space no wider than the [X, W, P] basis: dense (A_H, M_H)
    PASE_TRY(small_sygv(h, (int)NH, m, w.AHd, (int)NH, w.MHd, (int)NH, lam, w.CH, m, w.status));
    PASE_TRY(launch_ctl_status(h, w.status, true));
    PASE_TRY(launch_ctl_put(h, w.ci + CI_AUG_IT, 1, true, nullptr, 0.0));
  } else {
    PASE_CUDA(cudaMemsetAsync(w.S, 0, sizeof(double) * (NH + m) * m3, h->stream));
    PASE_TRY(launch_hash_fill(h, NH, m, m3, 12345u, w.S));
    BlockOp op{NH, 1, nullptr, nullptr, nullptr, nullptr};
    PASE_TRY(block_eigensolver(h, op, lam, nullptr, 1e-12, 10 * h->opt.aug_max_iter, m));
    PASE_TRY(launch_copy_cols(h, NH, m, w.S, m3, w.CH, m));
  }
  PASE_TRY(launch_csr<double>(h, CSR_MV, m, h->Pd, h->Pd.val, nullptr, w.CH, nullptr, nullptr, nullptr, nullptr,
                              0.0, U, nullptr, nullptr, nullptr));
  return PASE_OK;
}
static int coarse_start(pase_ctx* h, double* U, double* lam) {
  if (h->NH < h->w.m) return fail(PASE_ERR_INVALID_ARG, "coarse start needs N_H >= m");
  auto rec = [=]() -> int { return record_coarse_start(h, U, lam); };
  if (recording(h)) return rec();
  const std::vector<uint64_t> key = {key_of(U), key_of(lam)};
  if (!h->g_start.exec || h->g_start.key != key) {
    PASE_TRY(graph_record(h, h->g_start, rec));
    h->g_start.key = key;
  }
  return graph_launch(h, h->g_start);
}

// One outer iteration after the residual has been formed in w.R (or with W = U when
// do_solve is false): (a) (b) (c) (d); U and lam are overwritten.  Inside a recording
// step (a) is recorded in place (its own graph is for eager solves).
static int iterate_body(pase_ctx* h, double* U, double* lam, bool do_solve, cudaEvent_t* ev, bool graphed = false) {
  Work& w = h->w;
  const size_t nm = (size_t)h->N * w.m;
  if (recording(h)) ev = nullptr;
  if (ev) PASE_CUDA(cudaEventRecord(ev[0], h->stream));
  if (do_solve)
    PASE_TRY(graphed && !recording(h) ? step_linear_solve_graphed(h, U, w.W) : step_linear_solve(h, U, w.W));
  else PASE_CUDA(cudaMemcpyAsync(w.W, U, sizeof(double) * nm, cudaMemcpyDeviceToDevice, h->stream));
  if (ev) PASE_CUDA(cudaEventRecord(ev[1], h->stream));
  PASE_TRY(step_project(h, w.W, w.aH, w.bH, w.GA, w.GM));
  if (ev) PASE_CUDA(cudaEventRecord(ev[2], h->stream));
  PASE_TRY(step_augmented_eig(h, w.aH, w.bH, w.GA, w.GM, lam, w.CH, w.CW));
  if (ev) PASE_CUDA(cudaEventRecord(ev[3], h->stream));
  PASE_TRY(step_prolongate(h, w.W, w.CH, w.CW, U));
  if (ev) PASE_CUDA(cudaEventRecord(ev[4], h->stream));
  return PASE_OK;
}

// An error the device control block holds (cleared here): NaN, a start block that is not
// B-independent, or a double-float range flag.
static int ctl_error(pase_ctx* h, int err) {
  PASE_CUDA(cudaMemsetAsync(h->w.ci + CI_ERR, 0, sizeof(int), h->stream));
  if (err == kCtlErrDfRange) {
    PASE_CUDA(cudaMemsetAsync(h->w.df_flag, 0, sizeof(int), h->stream));
    return fail(PASE_ERR_NAN, "a block entry above 2^100 (or not finite) met the double-float products; "
                              "set spmm_df64 = 0 for such data");
  }
  if (err == PASE_ERR_NOT_SPD) return fail(err, "block eigensolver: start block is not B-independent");
  if (err == PASE_ERR_NAN) return fail(err, "NaN in an eigen-residual");
  if (err == PASE_ERR_TIMEOUT) return fail(err, "a recorded loop reached its pass limit");
  return fail(err, "device-side error");
}

// ------------------------------------------------------------------ batch scheme (§5)
// Batch boundaries (Alg. 7 step 2): batches of k pairs, a boundary moved up past any coarse
// eigenvalue within a relative gap of its predecessor, so that no cluster of the coarse
// spectrum is split between two batches.
static std::vector<std::pair<int, int>> batch_bounds(const std::vector<double>& lamH, int nev, int k) {
  std::vector<std::pair<int, int>> out;
  int m0 = 0;
  while (m0 < nev) {
    int e = std::min(nev, m0 + k);
    while (e < nev && lamH[e] - lamH[e - 1] <= 1e-3 * lamH[e]) ++e;
    out.push_back({m0, e});
    m0 = e;
  }
  return out;
}

static int batch_alloc(pase_ctx* h, int nev, int m) {
  auto& b = h->bb;
  if (b.AHd && b.nev >= nev && b.m == m) return PASE_OK;
  const int64_t NH = h->NH;
  b.nev = nev;
  b.m = m;
  b.top = nev + m;
  b.n = (int)NH + m;
  b.kk = std::min(b.n, nev + 3 * m);
  b.nw = std::min(2 * m, b.kk);
  PASE_TRY(dev_alloc_t(h, &b.AHd, (size_t)NH * NH));
  PASE_TRY(dev_alloc_t(h, &b.MHd, (size_t)NH * NH));
  PASE_TRY(dev_alloc_t(h, &b.CHc, (size_t)NH * b.top));
  PASE_TRY(dev_alloc_t(h, &b.lamH, (size_t)b.top));
  PASE_TRY(dev_alloc_t(h, &b.Ad, (size_t)b.n * b.n));
  PASE_TRY(dev_alloc_t(h, &b.Bd, (size_t)b.n * b.n));
  PASE_TRY(dev_alloc_t(h, &b.Cw, (size_t)b.n * b.kk));
  PASE_TRY(dev_alloc_t(h, &b.lamw, (size_t)b.kk));
  PASE_TRY(dev_alloc_t(h, &b.Cc, (size_t)b.n * b.nw));
  PASE_TRY(dev_alloc_t(h, &b.Rm, (size_t)b.nw * m));
  PASE_TRY(dev_alloc_t(h, &b.Rt, (size_t)m * b.nw));
  PASE_TRY(dev_alloc_t(h, &b.Rt2, (size_t)m * b.nw));
  PASE_TRY(dev_alloc_t(h, &b.S, (size_t)m * m));
  PASE_TRY(dev_alloc_t(h, &b.comp, (size_t)b.nw));
  PASE_TRY(dev_alloc_t(h, &b.idx, (size_t)std::max(b.nw, m)));
  b.eig_doubles = std::max(small_sygv_work_doubles((int)NH, b.top), small_sygv_work_doubles(b.n, b.kk)) + 64;
  PASE_TRY(dev_alloc_t(h, &b.eig, b.eig_doubles));
  return PASE_OK;
}

// small_sygv on the batch workspace (the handle's own is sized for 3m)
static int batch_sygv(pase_ctx* h, int n, int k, const double* A, const double* B, double* lam, double* C) {
  Work& w = h->w;
  double* keep = w.eigwork;
  const size_t keep_n = w.eigwork_doubles;
  w.eigwork = h->bb.eig;
  w.eigwork_doubles = h->bb.eig_doubles;
  const int rc = small_sygv(h, n, k, A, n, B, n, lam, C, k, w.status);
  w.eigwork = keep;
  w.eigwork_doubles = keep_n;
  PASE_TRY(rc);
  PASE_TRY(sync_small(h, nullptr, 0, w.status, 1));
  if (w.h_status[0] != 0) return fail(PASE_ERR_NOT_SPD, "batch scheme: dense generalized eigensolve failed");
  return PASE_OK;
}

static int upload_ints(pase_ctx* h, const std::vector<int>& v, int* d) {
  PASE_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, h->stream));
  return PASE_OK;
}

// the augmented pencil of Alg. 7 step (d), dense: [[A_H, aH], [aH^T, GA]], [[M_H, bH], [bH^T, GM]]
static int batch_assemble(pase_ctx* h) {
  auto& b = h->bb;
  Work& w = h->w;
  const int64_t NH = h->NH, n = b.n;
  const int m = w.m;
  const double* src[2][3] = {{b.AHd, w.aH, w.GA}, {b.MHd, w.bH, w.GM}};
  double* dst[2] = {b.Ad, b.Bd};
  for (int q = 0; q < 2; ++q) {
    PASE_TRY(launch_geam(h, NH, (int)NH, 1.0, src[q][0], NH, 0.0, src[q][0], NH, dst[q], n));
    PASE_TRY(launch_copy_cols(h, NH, m, src[q][1], m, dst[q] + NH, (int)n));
    PASE_TRY(launch_transpose(h, NH, m, src[q][1], m, dst[q] + NH * n, n));
    PASE_TRY(launch_copy_cols(h, m, m, src[q][2], m, dst[q] + NH * n + NH, (int)n));
  }
  return PASE_OK;
}

// ------------------------------------------------------------------ the solve loop
// Default block width: nev plus max(4, nev/10) guard columns, rounded up to 8.
static int default_block(int nev, int m) {
  if (m != 0) return m;
  const int g = nev + std::max(4, (nev + 9) / 10);
  return (g + 7) / 8 * 8;
}

// Alg. 3 step 7 (post_solve): A_h u = lambda M_h u-hat from the Rayleigh-Ritz block u-hat
// (its residual is in w.R), then the residual of the new block for the next step 3.
static int post_solve_step(pase_ctx* h) {
  Work& w = h->w;
  PASE_TRY(recording(h) ? step_linear_solve(h, w.U, w.W) : step_linear_solve_graphed(h, w.U, w.W));
  PASE_CUDA(cudaMemcpyAsync(w.U, w.W, sizeof(double) * h->N * w.m, cudaMemcpyDeviceToDevice, h->stream));
  return step_residual(h, w.U, w.lam, w.R);
}

// The start of a solve: the given block, or the coarse start of Alg. 3 steps 1-2.  With
// a given block the first iteration skips step (a) (W = U) and its inner tolerance is
// max(aug_tol, 1e-6) under the adaptive rule.
static int solve_start(pase_ctx* h, const double* dU0) {
  Work& w = h->w;
  PASE_TRY(launch_ctl_init(h));
  if (!dU0) return coarse_start(h, w.U, w.lam);
  PASE_CUDA(cudaMemcpyAsync(w.U, dU0, sizeof(double) * h->N * w.m, cudaMemcpyDeviceToDevice, h->stream));
  return launch_ctl_put(h, nullptr, 0, false, w.cd + CD_AUG_TOL,
                        h->opt.aug_adaptive ? std::max(h->opt.aug_tol, 1e-6) : h->opt.aug_tol);
}

// The whole solve, recorded (graph_solve): the start, the outer loop as a WHILE node
// whose test is k_ctl_outer_check (§6 stopping rule, max_iter, pending errors), the
// iteration under an IF node, and the copies of the result.
static int record_solve(pase_ctx* h, int nev, double tol, const double* dU0, double* dl, double* dU) {
  Work& w = h->w;
  PASE_TRY(solve_start(h, dU0));
  if (dU0) {
    PASE_TRY(iterate_body(h, w.U, w.lam, false, nullptr));
    PASE_TRY(launch_ctl_put(h, w.ci + CI_ITER, 1, true, nullptr, 0.0));
  }
  PASE_TRY(launch_ctl_put(h, w.ci + CI_OUT_CONT, 1, false, nullptr, 0.0));
  PASE_TRY(cond_node(h, true, w.ci + CI_OUT_CONT, [&]() -> int {
    PASE_TRY(step_residual(h, w.U, w.lam, w.R));
    PASE_TRY(launch_ctl_outer_check(h, nev, tol));
    return cond_node(h, false, w.ci + CI_OUT_GO, [&]() -> int {
      if (h->opt.post_solve)
        PASE_TRY(cond_node(h, false, w.ci + CI_POST, [&]() -> int { return post_solve_step(h); }));
      PASE_TRY(iterate_body(h, w.U, w.lam, true, nullptr));
      return launch_ctl_put(h, w.ci + CI_ITER, 1, true, nullptr, 0.0);
    });
  }, h->opt.max_iter + 2));
  PASE_CUDA(cudaMemcpyAsync(dl, w.lam, w.m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  PASE_CUDA(cudaMemcpyAsync(dU, w.U, sizeof(double) * h->N * w.m, cudaMemcpyDeviceToDevice, h->stream));
  return PASE_OK;
}

// What a recorded solve depends on besides the handle's fixed buffers.
static std::vector<uint64_t> solve_key(pase_ctx* h, int nev, double tol, const void* dU0, const void* dl,
                                       const void* dU) {
  return {(uint64_t)nev, key_of(tol), key_of(dU0), key_of(dl), key_of(dU), (uint64_t)h->aug_nconv,
          (uint64_t)sm_active(h), (uint64_t)h->opt.smoother};
}

// Statistics and status of a solve from the control block (read by sync_ctl).
static int solve_outcome(pase_ctx* h, pase_stats* st) {
  const Work& w = h->w;
  st->iterations = w.h_ci[CI_ITER];
  st->converged = w.h_ci[CI_CONV];
  st->max_residual = w.h_cd[CD_WORST];
  st->aug_iterations = w.h_ci[CI_AUG_IT];
  if (w.h_ci[CI_ERR]) return ctl_error(h, w.h_ci[CI_ERR]);
  if (w.h_ci[CI_MAXED]) return fail(PASE_ERR_NOT_CONVERGED, "maximum number of iterations reached");
  return PASE_OK;
}

// The solve driven from the host, one outer iteration at a time (per-phase timing): the
// same tests as the recorded solve, read back once per iteration; step (c) is a graph
// launch.
static int solve_stepwise(pase_ctx* h, int nev, double tol, const double* dU0, pase_stats* st) {
  Work& w = h->w;
  cudaEvent_t ev[6];
  for (auto& e : ev) PASE_CUDA(cudaEventCreate(&e));
  struct EvFree {
    cudaEvent_t* e;
    ~EvFree() {
      for (int i = 0; i < 6; ++i) cudaEventDestroy(e[i]);
    }
  } evfree{ev};
  PASE_TRY(solve_start(h, dU0));
  bool skip_test = dU0 != nullptr;  // the given block's first iteration has no test
  for (;;) {
    if (!skip_test) {
      PASE_CUDA(cudaEventRecord(ev[0], h->stream));
      PASE_TRY(step_residual(h, w.U, w.lam, w.R));
      PASE_CUDA(cudaEventRecord(ev[5], h->stream));
      PASE_TRY(launch_ctl_outer_check(h, nev, tol));
      PASE_TRY(sync_ctl(h));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[0], ev[5]);
      st->phase_ms[4] += ms;
      const int rc = solve_outcome(h, st);
      if (h->opt.verbose)
        fprintf(stderr, "[pase] iter %d  max relres(first %d) %.3e  aug_iters %d\n", st->iterations, nev,
                st->max_residual, st->aug_iterations);
      if (rc != PASE_OK) return rc;
      if (!w.h_ci[CI_OUT_GO]) return PASE_OK;
      if (w.h_ci[CI_POST]) {
        PASE_CUDA(cudaEventRecord(ev[0], h->stream));
        PASE_TRY(post_solve_step(h));
        PASE_CUDA(cudaEventRecord(ev[1], h->stream));
        PASE_CUDA(cudaEventSynchronize(ev[1]));
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        st->phase_ms[0] += ms;
      }
    }
    PASE_TRY(iterate_body(h, w.U, w.lam, !skip_test, ev, true));
    skip_test = false;
    PASE_TRY(launch_ctl_put(h, w.ci + CI_ITER, 1, true, nullptr, 0.0));
    PASE_CUDA(cudaEventSynchronize(ev[4]));
    for (int p = 0; p < 4; ++p) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[p], ev[p + 1]);
      st->phase_ms[p] += ms;
    }
  }
}


// ------------------------------------------------------------------ batched solve, one graph
// All handles distinct, set up, with graph_solve, on the current device.
static bool batch_graph_ok(pase_ctx* const* hs, int count) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !hs[i]->ready || !hs[i]->opt.graph_solve || hs[i]->device != dev) return false;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return false;
  }
  return true;
}

// Every problem's whole solve (as record_solve) is one branch of a single graph, launched
// once; the graph is kept by the first handle and reused while the handles, sizes and
// buffers stay the same.
static int solve_batched_graph(pase_ctx* const* hs, int count, const int* nev, const double* tol, const int* m,
                               const double* const* U0, double* const* lambda, double* const* U, pase_stats* st) {
  pase_ctx* h0 = hs[0];
  std::vector<std::unique_ptr<Stage>> sg(count);
  std::vector<const void*> dU0(count);
  std::vector<void*> dl(count), dU(count);
  std::vector<uint64_t> key;
  std::vector<int64_t> l0(count);
  auto t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < count; ++i) {
    pase_ctx* h = hs[i];
    const int mi = default_block(nev[i], m ? m[i] : 0);
    if (nev[i] < 1 || !(tol[i] > 0.0) || !lambda[i] || !U[i] || mi <= nev[i])
      return fail(PASE_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": bad arguments");
    PASE_TRY(reserve(h, mi));
    const double* u0 = U0 ? U0[i] : nullptr;
    if (!u0 && h->NH < mi) return fail(PASE_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": coarse start needs N_H >= m");
    sg[i].reset(new Stage(h));
    const size_t nm = (size_t)h->N * mi * sizeof(double);
    PASE_TRY(sg[i]->in(u0, nm, &dU0[i]));
    PASE_TRY(sg[i]->out(lambda[i], mi * sizeof(double), &dl[i]));
    PASE_TRY(sg[i]->out(U[i], nm, &dU[i]));
    h->aug_nconv = std::min(mi, nev[i] + std::max(1, (mi - nev[i]) / 2));
    key.push_back(h->serial);
    for (uint64_t k : solve_key(h, nev[i], tol[i], dU0[i], dl[i], dU[i])) key.push_back(k);
    l0[i] = h->launches;
  }
  if (!h0->batch_exec || h0->batch_key != key) {
    if (h0->batch_exec) cudaGraphExecDestroy(h0->batch_exec);
    h0->batch_exec = nullptr;
    h0->batch_key.clear();
    PASE_TRY(batch_record(hs, count, [&](int i) -> int {
      return record_solve(hs[i], nev[i], tol[i], (const double*)dU0[i], (double*)dl[i], (double*)dU[i]);
    }, &h0->batch_exec));
    h0->batch_key = key;
  }
  // order: the staged inputs of every handle, the graph on the first handle's stream, then
  // the copies back on every handle's stream
  cudaEvent_t e = nullptr;
  PASE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  struct EvFree {
    cudaEvent_t e;
    ~EvFree() { cudaEventDestroy(e); }
  } evfree{e};
  for (int i = 1; i < count; ++i) {
    PASE_CUDA(cudaEventRecord(e, hs[i]->stream));
    PASE_CUDA(cudaStreamWaitEvent(h0->stream, e, 0));
  }
  PASE_CUDA(cudaGraphLaunch(h0->batch_exec, h0->stream));
  h0->graph_launches++;
  PASE_CUDA(cudaEventRecord(e, h0->stream));
  for (int i = 0; i < count; ++i) {
    hs[i]->launches += hs[i]->g_batch.top_kernels;
    hs[i]->replayed += hs[i]->g_batch.top_kernels;
    if (i) PASE_CUDA(cudaStreamWaitEvent(hs[i]->stream, e, 0));
  }
  int rc = PASE_OK;
  for (int i = 0; i < count; ++i) {
    pase_ctx* h = hs[i];
    PASE_TRY(sg[i]->finish());
    PASE_TRY(sync_ctl(h));
    pase_stats s;
    memset(&s, 0, sizeof(s));
    int ri = solve_outcome(h, &s);
    h->aug_nconv = 0;
    if (ri == PASE_OK && sm_active(h)) ri = sm_check_timeout(h);
    if (ri == PASE_OK) ri = tc_check(h);
    s.kernel_launches = (int)(h->launches - l0[i]);
    s.graph_launches = i == 0 ? 1 : 0;
    if (st) st[i] = s;
    if (ri != PASE_OK && ri != PASE_ERR_NOT_CONVERGED && (rc == PASE_OK || rc == PASE_ERR_NOT_CONVERGED)) {
      rc = fail(ri, "problem " + std::to_string(i) + ": " + pase_last_error());
    } else if (ri == PASE_ERR_NOT_CONVERGED && rc == PASE_OK) {
      rc = PASE_ERR_NOT_CONVERGED;
    }
  }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st)
    for (int i = 0; i < count; ++i) st[i].solve_ms = ms;
  if (rc == PASE_ERR_NOT_CONVERGED) pase::set_error("some problems reached max_iter");
  return rc;
}

}  // namespace pase

using namespace pase;

// ====================================================================== C ABI
extern "C" {

void pase_default_options(pase_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = PASE_PREC_FP64;
  o->linear_solver = PASE_SOLVER_VCYCLE;
  o->inner_steps = 2;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = 2.0 / 3.0;
  o->coarse_level = -1;
  o->max_iter = 100;
  o->aug_max_iter = 60;
  o->aug_tol = 1e-12;
  o->aug_adaptive = 1;
  o->verbose = 0;
  o->use_graphs = 1;
  o->autotune = 1;
  o->smoother = PASE_SMOOTHER_JACOBI;
  o->split_gemm = 1;
  o->stencil = 1;
  o->post_solve = 0;
  o->aug_transform = PASE_AUG_PLAIN;
  o->spmm_df64 = 1;
  o->graph_solve = 0;
  o->aug_factor = 1e-4;
  o->sygv_tridiag = -1;
  o->sygv_cholesky = -1;
}

const char* pase_status_string(int code) {
  switch (code) {
    case PASE_OK: return "ok";
    case PASE_ERR_INVALID_ARG: return "invalid argument";
    case PASE_ERR_SHAPE_MISMATCH: return "shape mismatch";
    case PASE_ERR_PATTERN_MISMATCH: return "sparsity pattern mismatch";
    case PASE_ERR_NOT_SPD: return "matrix not symmetric positive definite";
    case PASE_ERR_NAN: return "NaN or Inf encountered";
    case PASE_ERR_NOT_CONVERGED: return "not converged";
    case PASE_ERR_TIMEOUT: return "device wait timed out";
    case PASE_ERR_CUDA: return "CUDA error";
    case PASE_ERR_OUT_OF_MEMORY: return "out of device memory";
    case PASE_ERR_STATE: return "call out of order";
    case PASE_ERR_BAD_CSR: return "malformed CSR matrix";
    default: return "unknown status";
  }
}

const char* pase_last_error(void) { return pase::last_error_cstr(); }

int pase_create(pase_handle* out, const pase_options* opt, void* stream) {
  if (!out) return fail(PASE_ERR_INVALID_ARG, "pase_create: null handle pointer");
  *out = nullptr;
  pase_ctx* h = new (std::nothrow) pase_ctx();
  if (!h) return fail(PASE_ERR_OUT_OF_MEMORY, "pase_create: host allocation failed");
  if (opt) h->opt = *opt;
  else pase_default_options(&h->opt);
  const pase_options& o = h->opt;
  if ((o.precision != PASE_PREC_FP64 && o.precision != PASE_PREC_MIXED) || o.inner_steps < 1 || o.nu1 < 0 ||
      o.linear_solver < PASE_SOLVER_VCYCLE || o.linear_solver > PASE_SOLVER_MGCG ||
      (o.smoother != PASE_SMOOTHER_JACOBI && o.smoother != PASE_SMOOTHER_LEARNED) ||
      (o.post_solve != 0 && o.post_solve != 1) || (o.graph_solve != 0 && o.graph_solve != 1) ||
      (o.stencil_columns != 0 && o.stencil_columns != 2 && o.stencil_columns != 4) ||
      o.sygv_tridiag < -1 || o.sygv_tridiag > 2 || o.sygv_cholesky < -1 || o.sygv_cholesky > 1 ||
      o.graph_pass_limit < 0 || !(o.aug_factor > 0.0 && o.aug_factor <= 1.0) ||
      o.aug_transform < PASE_AUG_PLAIN ||
      o.aug_transform > PASE_AUG_PRECOND_BA ||
      o.nu2 < 0 || !(o.omega > 0.0 && o.omega < 2.0) || o.max_iter < 1 || o.aug_max_iter < 1 ||
      !(o.aug_tol > 0.0)) {
    delete h;
    return fail(PASE_ERR_INVALID_ARG, "pase_create: invalid options");
  }
  h->stream = (cudaStream_t)stream;
  static std::atomic<uint64_t> serials(0);
  h->serial = ++serials;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(PASE_ERR_CUDA, "pase_create: no CUDA device");
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess && sms > 0)
    h->num_sms = sms;
  *out = h;
  return PASE_OK;
}

int pase_destroy(pase_handle h) {
  if (!h) return PASE_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->ls_graph) cudaGraphExecDestroy(h->ls_graph);
  for (pase::GraphRec* g : {&h->g_stepc, &h->g_start, &h->g_solve, &h->g_batch}) pase::graph_free(*g);
  if (h->batch_exec) cudaGraphExecDestroy(h->batch_exec);
  for (cudaStream_t s : h->cap_streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  sm_free(h);
  for (void* p : h->allocations) cudaFree(p);
  if (h->w.h_small) cudaFreeHost(h->w.h_small);
  if (h->w.h_status) cudaFreeHost(h->w.h_status);
  if (h->w.h_ci) cudaFreeHost(h->w.h_ci);
  if (h->w.h_cd) cudaFreeHost(h->w.h_cd);
  delete h;
  return PASE_OK;
}

int pase_setup(pase_handle h, const pase_csr* A_h, const pase_csr* M_h, int n_interp, const pase_csr* P,
               const pase_csr* A_H, const pase_csr* M_H) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "pase_setup: null handle");
  if (h->ready) return fail(PASE_ERR_STATE, "pase_setup: handle already set up");
  if (n_interp < 1 || !P) return fail(PASE_ERR_INVALID_ARG, "pase_setup: need at least one interpolation matrix");
  HostCSR A0, M0, AHc, MHc;
  PASE_TRY(csr_from_abi(A_h, A0, "A_h"));
  PASE_TRY(csr_from_abi(M_h, M0, "M_h"));
  const bool coarse_given = A_H != nullptr || M_H != nullptr;
  if (coarse_given) {
    PASE_TRY(csr_from_abi(A_H, AHc, "A_H"));
    PASE_TRY(csr_from_abi(M_H, MHc, "M_H"));
  }
  std::vector<HostCSR> Pc(n_interp);
  for (int k = 0; k < n_interp; ++k) PASE_TRY(csr_from_abi(&P[k], Pc[k], "P"));
  if (A0.nrows != A0.ncols || A0.nrows == 0) return fail(PASE_ERR_SHAPE_MISMATCH, "A_h must be square and non-empty");
  if (!same_pattern(A0, M0)) return fail(PASE_ERR_PATTERN_MISMATCH, "A_h and M_h must share one sparsity pattern");
  if (coarse_given && !same_pattern(AHc, MHc))
    return fail(PASE_ERR_PATTERN_MISMATCH, "A_H and M_H must share one sparsity pattern");
  int c = h->opt.coarse_level < 0 ? n_interp : h->opt.coarse_level;
  if (c < 1 || c > n_interp) return fail(PASE_ERR_INVALID_ARG, "coarse_level out of range");
  int64_t rows = A0.nrows;
  for (int k = 0; k < n_interp; ++k) {
    if (Pc[k].nrows != rows || Pc[k].ncols <= 0) return fail(PASE_ERR_SHAPE_MISMATCH, "P chain shapes do not match");
    rows = Pc[k].ncols;
  }
  // levels
  h->L = n_interp + 1;
  h->coarse_level = c;
  std::vector<HostCSR> Al(h->L);
  Al[0] = A0;
  for (int k = 0; k < n_interp; ++k) Al[k + 1] = csr_galerkin(Pc[k], Al[k]);
  if (!coarse_given) {  // the coarse pencil of nested spaces: Galerkin products through the chain
    AHc = Al[c];
    MHc = M0;
    for (int k = 0; k < c; ++k) MHc = csr_galerkin(Pc[k], MHc);
    if (!same_pattern(AHc, MHc)) return fail(PASE_ERR_PATTERN_MISMATCH, "Galerkin A_H and M_H patterns differ");
  }
  if (AHc.nrows != Al[c].nrows || AHc.ncols != Al[c].nrows)
    return fail(PASE_ERR_SHAPE_MISMATCH, "A_H does not match the size of the coarse level");
  const HostCSR& Ac = Al[h->L - 1];
  if (Ac.nrows > 8192) return fail(PASE_ERR_INVALID_ARG, "coarsest multigrid level too large for a dense solve (> 8192)");
  std::vector<double> cinv;
  if (!dense_spd_inverse(Ac, cinv)) return fail(PASE_ERR_NOT_SPD, "coarsest multigrid operator is not SPD");
  HostCSR Pd = Pc[0];
  for (int k = 1; k < c; ++k) Pd = csr_multiply(Pd, Pc[k]);
  const bool mixed = h->opt.precision == PASE_PREC_MIXED;
  h->N = A0.nrows;
  h->NH = AHc.nrows;
  h->lv.resize(h->L);
  for (int l = 0; l < h->L; ++l) {
    Level& L = h->lv[l];
    PASE_TRY(upload_csr(h, Al[l], L.A, mixed, false, nullptr));
    std::vector<double> dinv(Al[l].nrows);
    for (int64_t i = 0; i < Al[l].nrows; ++i) {
      double dg = 0.0;
      for (int64_t k = Al[l].rowptr[i]; k < Al[l].rowptr[i + 1]; ++k)
        if (Al[l].col[k] == i) dg = Al[l].val[k];
      if (!(dg > 0.0)) return fail(PASE_ERR_NOT_SPD, "non-positive diagonal entry in a multigrid level");
      dinv[i] = 1.0 / dg;
    }
    PASE_TRY(upload_vec(h, dinv, &L.dinv));
    if (mixed) {
      std::vector<float> d32(dinv.begin(), dinv.end());
      PASE_TRY(upload_vec(h, d32, &L.dinv32));
      if (h->opt.stencil) PASE_TRY(stencil_setup(h, Al[l], dinv, L.A));
      if (h->opt.stencil_columns) L.A.st_cw = h->opt.stencil_columns;
    }
    if (l < n_interp) {
      PASE_TRY(upload_csr(h, Pc[l], L.P, mixed, false, nullptr));
      PASE_TRY(upload_csr(h, csr_transpose(Pc[l]), L.PT, mixed, false, nullptr));
    }
  }
  {
    DevCSR Mtmp;
    PASE_TRY(upload_csr(h, M0, Mtmp, mixed, true, &h->lv[0].A));
    h->M0_val = Mtmp.val;
    h->M0_val32 = Mtmp.val32;
  }
  if (h->opt.spmm_df64) {  // hi = fl32(v), lo = fl32(v - hi) of the fine pencil's values
    const int64_t nz = A0.nnz();
    std::vector<float> hi(std::max<int64_t>(1, nz)), lo(std::max<int64_t>(1, nz));
    float** dst[4] = {&h->A0h, &h->A0l, &h->M0h, &h->M0l};
    for (int q = 0; q < 2; ++q) {
      const std::vector<double>& v = q == 0 ? A0.val : M0.val;
      for (int64_t k = 0; k < nz; ++k) {
        hi[k] = (float)v[k];
        lo[k] = (float)(v[k] - (double)hi[k]);
      }
      PASE_TRY(upload_vec(h, hi, dst[2 * q]));
      PASE_TRY(upload_vec(h, lo, dst[2 * q + 1]));
    }
  }
  PASE_TRY(upload_csr(h, Pd, h->Pd, false, false, nullptr));
  PASE_TRY(upload_csr(h, csr_transpose(Pd), h->PdT, false, false, nullptr));
  PASE_TRY(upload_csr(h, AHc, h->AH, false, false, nullptr));
  {
    DevCSR Mtmp;
    PASE_TRY(upload_csr(h, MHc, Mtmp, false, true, &h->AH));
    h->MH_val = Mtmp.val;
    std::vector<double> md(MHc.nrows, 0.0);
    for (int64_t i = 0; i < MHc.nrows; ++i) {
      for (int64_t k = MHc.rowptr[i]; k < MHc.rowptr[i + 1]; ++k)
        if (MHc.col[k] == i) md[i] = MHc.val[k];
      if (!(md[i] > 0.0)) return fail(PASE_ERR_NOT_SPD, "non-positive diagonal entry in M_H");
      md[i] = 1.0 / md[i];
    }
    PASE_TRY(upload_vec(h, md, &h->MH_dinv));
  }
  h->ncoarsest = Ac.nrows;
  PASE_TRY(upload_vec(h, cinv, &h->cinv));
  if (mixed) {
    std::vector<float> c32(cinv.begin(), cinv.end());
    PASE_TRY(upload_vec(h, c32, &h->cinv32));
  }
  PASE_CUDA(cudaDeviceSynchronize());
  h->ready = true;
  return PASE_OK;
}

int pase_reserve(pase_handle h, int m) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  return reserve(h, m);
}

static int check_m(pase_handle h, int m) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  return reserve(h, m);
}

int pase_residual(pase_handle h, int m, const double* U, const double* lambda, double* R, double* relres) {
  PASE_TRY(check_m(h, m));
  if (!U || !lambda) return fail(PASE_ERR_INVALID_ARG, "pase_residual: null input");
  Stage st(h);
  const size_t nm = (size_t)h->N * m * sizeof(double);
  const void *dU, *dl;
  void *dR, *drr;
  PASE_TRY(st.in(U, nm, &dU));
  PASE_TRY(st.in(lambda, m * sizeof(double), &dl));
  PASE_TRY(st.out(R, nm, &dR));
  PASE_TRY(st.out(relres, m * sizeof(double), &drr));
  PASE_TRY(step_residual(h, (const double*)dU, (const double*)dl, dR ? (double*)dR : h->w.R));
  if (drr) PASE_CUDA(cudaMemcpyAsync(drr, h->w.relres, m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  PASE_TRY(st.finish());
  return df_check(h);
}

int pase_linear_solve(pase_handle h, int m, const double* U, const double* lambda, const double* R, double* W) {
  PASE_TRY(check_m(h, m));
  if (!U || !lambda || !W) return fail(PASE_ERR_INVALID_ARG, "pase_linear_solve: null argument");
  Stage st(h);
  const size_t nm = (size_t)h->N * m * sizeof(double);
  const void *dU, *dl, *dRin;
  void* dW;
  PASE_TRY(st.in(U, nm, &dU));
  PASE_TRY(st.in(lambda, m * sizeof(double), &dl));
  PASE_TRY(st.in(R, nm, &dRin));
  PASE_TRY(st.out(W, nm, &dW));
  if (dRin) PASE_CUDA(cudaMemcpyAsync(h->w.R, dRin, nm, cudaMemcpyDeviceToDevice, h->stream));
  else PASE_TRY(step_residual(h, (const double*)dU, (const double*)dl, h->w.R));
  PASE_TRY(step_linear_solve(h, (const double*)dU, (double*)dW));
  return st.finish();
}

int pase_project(pase_handle h, int m, const double* W, double* aH, double* bH, double* GA, double* GM) {
  PASE_TRY(check_m(h, m));
  if (!W || !aH || !bH || !GA || !GM) return fail(PASE_ERR_INVALID_ARG, "pase_project: null argument");
  Stage st(h);
  const size_t nm = (size_t)h->N * m * sizeof(double), hm = (size_t)h->NH * m * sizeof(double),
               mm = (size_t)m * m * sizeof(double);
  const void* dW;
  void *da, *db, *dga, *dgm;
  PASE_TRY(st.in(W, nm, &dW));
  PASE_TRY(st.out(aH, hm, &da));
  PASE_TRY(st.out(bH, hm, &db));
  PASE_TRY(st.out(GA, mm, &dga));
  PASE_TRY(st.out(GM, mm, &dgm));
  PASE_TRY(step_project(h, (const double*)dW, (double*)da, (double*)db, (double*)dga, (double*)dgm));
  PASE_TRY(st.finish());
  return df_check(h);
}

int pase_augmented_eig(pase_handle h, int m, const double* aH, const double* bH, const double* GA,
                       const double* GM, double* lambda, double* C_H, double* C_W, int* aug_iters) {
  PASE_TRY(check_m(h, m));
  if (!aH || !bH || !GA || !GM || !lambda || !C_H || !C_W) return fail(PASE_ERR_INVALID_ARG, "pase_augmented_eig: null argument");
  Stage st(h);
  const size_t hm = (size_t)h->NH * m * sizeof(double), mm = (size_t)m * m * sizeof(double);
  const void *da, *db, *dga, *dgm;
  void *dl, *dch, *dcw;
  PASE_TRY(st.in(aH, hm, &da));
  PASE_TRY(st.in(bH, hm, &db));
  PASE_TRY(st.in(GA, mm, &dga));
  PASE_TRY(st.in(GM, mm, &dgm));
  PASE_TRY(st.out(lambda, m * sizeof(double), &dl));
  PASE_TRY(st.out(C_H, hm, &dch));
  PASE_TRY(st.out(C_W, mm, &dcw));
  Work& w = h->w;
  PASE_TRY(launch_ctl_put(h, w.ci + CI_AUG_IT, 0, false, w.cd + CD_AUG_TOL, h->opt.aug_tol));
  PASE_TRY(step_augmented_eig(h, (const double*)da, (const double*)db, (const double*)dga, (const double*)dgm,
                              (double*)dl, (double*)dch, (double*)dcw));
  PASE_TRY(st.finish());
  PASE_TRY(sync_ctl(h));
  if (w.h_ci[CI_ERR]) return ctl_error(h, w.h_ci[CI_ERR]);
  if (aug_iters) *aug_iters = w.h_ci[CI_AUG_IT];
  return PASE_OK;
}

int pase_prolongate(pase_handle h, int m, const double* W, const double* C_H, const double* C_W, double* U) {
  PASE_TRY(check_m(h, m));
  if (!W || !C_H || !C_W || !U) return fail(PASE_ERR_INVALID_ARG, "pase_prolongate: null argument");
  Stage st(h);
  const size_t nm = (size_t)h->N * m * sizeof(double), hm = (size_t)h->NH * m * sizeof(double),
               mm = (size_t)m * m * sizeof(double);
  const void *dW, *dch, *dcw;
  void* dU;
  PASE_TRY(st.in(W, nm, &dW));
  PASE_TRY(st.in(C_H, hm, &dch));
  PASE_TRY(st.in(C_W, mm, &dcw));
  PASE_TRY(st.out(U, nm, &dU));
  if (dU == dW) return fail(PASE_ERR_INVALID_ARG, "pase_prolongate: U must not alias W");
  PASE_TRY(step_prolongate(h, (const double*)dW, (const double*)dch, (const double*)dcw, (double*)dU));
  PASE_TRY(st.finish());
  return tc_check(h);
}

int pase_iterate(pase_handle h, int nev, int m, double* U, double* lambda, int do_linear_solve,
                 double* relres) {
  PASE_TRY(check_m(h, m));
  if (!U || !lambda || nev < 1 || nev > m) return fail(PASE_ERR_INVALID_ARG, "pase_iterate: bad argument");
  Stage st(h);
  const size_t nm = (size_t)h->N * m * sizeof(double);
  void *dU, *dl, *drr;
  PASE_TRY(st.out(U, nm, &dU, true));
  PASE_TRY(st.out(lambda, m * sizeof(double), &dl, true));
  PASE_TRY(st.out(relres, m * sizeof(double), &drr));
  h->aug_nconv = std::min(m, nev + std::max(1, (m - nev) / 2));
  Work& w = h->w;
  const double* dUc = (const double*)dU;
  if (do_linear_solve || drr) {
    PASE_TRY(step_residual(h, dUc, (const double*)dl, w.R));
    if (drr) PASE_CUDA(cudaMemcpyAsync(drr, w.relres, m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  }
  if (do_linear_solve && h->opt.aug_adaptive) PASE_TRY(launch_ctl_aug_tol(h, nev));
  else
    PASE_TRY(launch_ctl_put(h, nullptr, 0, false, w.cd + CD_AUG_TOL,
                            (!drr && h->opt.aug_adaptive) ? std::max(h->opt.aug_tol, 1e-6) : h->opt.aug_tol));
  const int rc = iterate_body(h, (double*)dU, (double*)dl, do_linear_solve != 0, nullptr, true);
  h->aug_nconv = 0;
  PASE_TRY(rc);
  PASE_TRY(st.finish());
  PASE_TRY(sync_ctl(h));
  if (w.h_ci[CI_ERR]) return ctl_error(h, w.h_ci[CI_ERR]);
  PASE_TRY(df_check(h));
  return tc_check(h);
}

int pase_spmm_am(pase_handle h, int m, const double* X, double* AX, double* MX) {
  PASE_TRY(check_m(h, m));
  if (!is_device_ptr(X) || !is_device_ptr(AX) || !is_device_ptr(MX))
    return fail(PASE_ERR_INVALID_ARG, "pase_spmm_am: device pointers required");
  PASE_TRY(fine_products(h, CSR_MV_AM, X, nullptr, AX, MX, nullptr));
  PASE_CUDA(cudaStreamSynchronize(h->stream));
  return df_check(h);
}

int pase_smooth(pase_handle h, int m, int sweeps, const double* B, double* X) {
  PASE_TRY(check_m(h, m));
  if (!B || !X || sweeps < 1) return fail(PASE_ERR_INVALID_ARG, "pase_smooth: bad argument");
  Stage st(h);
  const size_t nm = (size_t)h->N * m;
  const void* dB;
  void* dX;
  PASE_TRY(st.in(B, nm * sizeof(double), &dB));
  PASE_TRY(st.out(X, nm * sizeof(double), &dX, true));
  const Level& L0 = h->lv[0];
  Work& w = h->w;
  if (h->opt.precision == PASE_PREC_MIXED) {
    PASE_TRY(launch_f64_to_f32(h, (int64_t)nm, (const double*)dB, w.fb[0]));
    PASE_TRY(launch_f64_to_f32(h, (int64_t)nm, (const double*)dX, w.fx[0]));
    float *cur = w.fx[0], *other = w.ft1[0];
    for (int s = 0; s < sweeps; ++s) {
      PASE_TRY(launch_csr<float>(h, CSR_JACOBI, m, L0.A, L0.A.val32, nullptr, cur, nullptr, w.fb[0], L0.dinv32,
                                 nullptr, h->opt.omega, other, nullptr, nullptr, nullptr));
      std::swap(cur, other);
    }
    PASE_TRY(launch_f32_to_f64(h, (int64_t)nm, cur, (double*)dX));
  } else {
    double *cur = (double*)dX, *other = w.T1;
    for (int s = 0; s < sweeps; ++s) {
      PASE_TRY(launch_csr<double>(h, CSR_JACOBI, m, L0.A, L0.A.val, nullptr, cur, nullptr, (const double*)dB,
                                  L0.dinv, nullptr, h->opt.omega, other, nullptr, nullptr, nullptr));
      std::swap(cur, other);
    }
    if (cur != (double*)dX)
      PASE_CUDA(cudaMemcpyAsync(dX, cur, nm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  }
  return st.finish();
}

int pase_smoother_form(pase_handle h) {
  if (!h || !h->ready || h->lv.empty()) return 0;
  return (h->opt.stencil && h->lv[0].A.st_val && h->lv[0].A.st_use) ? h->lv[0].A.st_dim : 0;
}

int64_t pase_kernel_count(pase_handle h) { return h ? h->launches : 0; }

int pase_launch_counts(pase_handle h, int64_t* kernels, int64_t* kernels_in_graphs, int64_t* graph_launches) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  if (kernels) *kernels = h->launches;
  if (kernels_in_graphs) *kernels_in_graphs = h->replayed;
  if (graph_launches) *graph_launches = h->graph_launches;
  return PASE_OK;
}

int pase_time_kernel(pase_handle h, int kernel, int m, int reps, double* ms_per_launch) {
  PASE_TRY(check_m(h, m));
  if (reps < 1 || !ms_per_launch) return fail(PASE_ERR_INVALID_ARG, "pase_time_kernel: bad arguments");
  Work& w = h->w;
  const size_t nm = (size_t)h->N * m;
  const bool mixed = h->opt.precision == PASE_PREC_MIXED;
  if ((kernel == PASE_KERNEL_JACOBI_FP32 || kernel == PASE_KERNEL_JACOBI_FP32_CSR) && !mixed)
    return fail(PASE_ERR_STATE, "pase_time_kernel: the FP32 smoother needs a PASE_PREC_MIXED handle");
  if (kernel < 0 || kernel > PASE_KERNEL_SPMM_AM_DF64)
    return fail(PASE_ERR_INVALID_ARG, "pase_time_kernel: unknown kernel");
  if (kernel == PASE_KERNEL_PROLONG_SPLIT && !ts_gemm_split_ok(m, m, h->w.W, m, h->w.T1, m))
    return fail(PASE_ERR_INVALID_ARG, "pase_time_kernel: the split GEMM takes m <= 128");
  if (kernel == PASE_KERNEL_GRAM_SPLIT && !ts_gram2_split_ok(h->N, m, h->num_sms, h->w))
    return fail(PASE_ERR_INVALID_ARG, "pase_time_kernel: the split Gram takes m <= 128");
  // deterministic operands
  PASE_TRY(launch_hash_fill(h, h->N, m, m, 7u, w.W));
  PASE_TRY(launch_hash_fill(h, h->N, m, m, 8u, w.R));
  PASE_TRY(launch_hash_fill(h, m, m, m, 9u, w.CW));
  if (mixed) {
    PASE_TRY(launch_f64_to_f32(h, nm, w.W, w.fx[0]));
    PASE_TRY(launch_f64_to_f32(h, nm, w.R, w.fb[0]));
  }
  const int m3 = 3 * m;
  if (kernel == PASE_KERNEL_SYGV) {  // a generic symmetric-definite pair (distinct eigenvalues)
    PASE_TRY(ts_gram(h, h->N, m, m, w.R, m, w.R, m, w.Gq, m3, true));
    PASE_TRY(ts_gram(h, h->N, m, m, w.W, m, w.W, m, w.Gb, m3, true));
  }
  if (kernel == PASE_KERNEL_SYGV3) {  // the Rayleigh-Ritz size of the step-(c) solver
    const int64_t nc = h->NH + m;
    PASE_TRY(launch_hash_fill(h, nc, m3, m3, 10u, w.S));
    PASE_TRY(launch_hash_fill(h, nc, m3, m3, 11u, w.AS));
    PASE_TRY(ts_gram(h, nc, m3, m3, w.AS, m3, w.AS, m3, w.Gq, m3, true));
    PASE_TRY(ts_gram(h, nc, m3, m3, w.S, m3, w.S, m3, w.Gb, m3, true));
  }
  const Level& L0 = h->lv[0];
  auto once = [&]() -> int {
    switch (kernel) {
      case PASE_KERNEL_SPMM_AM_FP64:
        return launch_csr<double>(h, CSR_MV_AM, m, L0.A, L0.A.val, h->M0_val, w.W, nullptr, nullptr, nullptr,
                                  nullptr, 0.0, w.T1, w.T2, nullptr, nullptr);
      case PASE_KERNEL_JACOBI_FP64:
        return launch_csr<double>(h, CSR_JACOBI, m, L0.A, L0.A.val, nullptr, w.W, nullptr, w.R, L0.dinv, nullptr,
                                  h->opt.omega, w.T1, nullptr, nullptr, nullptr);
      case PASE_KERNEL_JACOBI_FP32:
        return launch_csr<float>(h, CSR_JACOBI, m, L0.A, L0.A.val32, nullptr, w.fx[0], nullptr, w.fb[0], L0.dinv32,
                                 nullptr, h->opt.omega, w.ft1[0], nullptr, nullptr, nullptr);
      case PASE_KERNEL_JACOBI_FP32_CSR: {  // the CSR kernel even where the structured one applies
        DevCSR A = L0.A;
        A.st_val = nullptr;
        return launch_csr<float>(h, CSR_JACOBI, m, A, L0.A.val32, nullptr, w.fx[0], nullptr, w.fb[0], L0.dinv32,
                                 nullptr, h->opt.omega, w.ft1[0], nullptr, nullptr, nullptr);
      }
      case PASE_KERNEL_GRAM_FP64:
        return ts_gram(h, h->N, m, m, w.W, m, w.R, m, w.GA, m, true);
      case PASE_KERNEL_FMA_FP64:
        return launch_fma_fp64(h, w.smallvec);
      case PASE_KERNEL_SPMM_AM_DF64:
        if (!use_df64(h)) return fail(PASE_ERR_STATE, "pase_time_kernel: the handle has spmm_df64 = 0");
        return fine_products(h, CSR_MV_AM, w.W, nullptr, w.T1, w.T2, nullptr);
      case PASE_KERNEL_PROLONG_FP64:
        return ts_gemm(h, h->N, m, m, 1.0, w.W, m, w.CW, m, 0.0, w.T1, m);
      case PASE_KERNEL_PROLONG_SPLIT:
        return ts_gemm_split(h, h->N, m, m, w.W, m, w.CW, m, w.T1, m, h->tc_err);
      case PASE_KERNEL_GRAM_SPLIT:
        return ts_gram2_split(h, h->N, m, w.W, w.R, w.W, w.GA, w.GM, m, w.colexp, h->tc_err);
      case PASE_KERNEL_SYGV:
        return small_sygv(h, m, m, w.Gq, m3, w.Gb, m3, w.smallvec, w.Cs, m, w.status);
      case PASE_KERNEL_SYGV3:
        return small_sygv(h, m3, m, w.Gq, m3, w.Gb, m3, w.smallvec, w.Cs, m, w.status);
    }
    return PASE_OK;
  };
  for (int i = 0; i < 2; ++i) PASE_TRY(once());
  cudaEvent_t e0, e1;
  PASE_CUDA(cudaEventCreate(&e0));
  PASE_CUDA(cudaEventCreate(&e1));
  PASE_CUDA(cudaEventRecord(e0, h->stream));
  for (int i = 0; i < reps; ++i) PASE_TRY(once());
  PASE_CUDA(cudaEventRecord(e1, h->stream));
  PASE_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  PASE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_per_launch = (double)ms / reps;
  return tc_check(h);
}

int pase_solve(pase_handle h, int nev, double tol, int m, const double* U0, double* lambda, double* U,
               pase_stats* stp) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  if (!h->ready) return fail(PASE_ERR_STATE, "pase_setup has not completed");
  if (nev < 1 || !(tol > 0.0) || !lambda || !U) return fail(PASE_ERR_INVALID_ARG, "pase_solve: bad arguments");
  m = default_block(nev, m);
  if (m <= nev) return fail(PASE_ERR_INVALID_ARG, "pase_solve: m must exceed nev");
  PASE_TRY(reserve(h, m));
  if (!U0 && h->NH < m) return fail(PASE_ERR_INVALID_ARG, "coarse start needs N_H >= m");
  Work& w = h->w;
  pase_stats st;
  memset(&st, 0, sizeof(st));
  const int64_t launches0 = h->launches, graphs0 = h->graph_launches;
  Stage sg(h);
  const size_t nm = (size_t)h->N * m * sizeof(double);
  const void* dU0;
  void *dl, *dU;
  PASE_TRY(sg.in(U0, nm, &dU0));
  PASE_TRY(sg.out(lambda, m * sizeof(double), &dl));
  PASE_TRY(sg.out(U, nm, &dU));
  h->aug_nconv = std::min(m, nev + std::max(1, (m - nev) / 2));
  auto t0 = std::chrono::steady_clock::now();
  int rc = PASE_OK;
  if (h->opt.graph_solve) {
    // the whole solve is one graph launch
    const std::vector<uint64_t> key = solve_key(h, nev, tol, dU0, dl, dU);
    if (!h->g_solve.exec || h->g_solve.key != key) {
      PASE_TRY(graph_record(h, h->g_solve, [&]() -> int {
        return record_solve(h, nev, tol, (const double*)dU0, (double*)dl, (double*)dU);
      }));
      h->g_solve.key = key;
    }
    PASE_TRY(graph_launch(h, h->g_solve));
    PASE_TRY(sg.finish());
    PASE_TRY(sync_ctl(h));
    rc = solve_outcome(h, &st);
  } else {
    rc = solve_stepwise(h, nev, tol, (const double*)dU0, &st);
    if (rc == PASE_OK || rc == PASE_ERR_NOT_CONVERGED) {
      PASE_CUDA(cudaMemcpyAsync(dl, w.lam, m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      PASE_CUDA(cudaMemcpyAsync(dU, w.U, nm, cudaMemcpyDeviceToDevice, h->stream));
    }
    PASE_TRY(sg.finish());
    PASE_TRY(sync_ctl(h));
    st.aug_iterations = w.h_ci[CI_AUG_IT];
  }
  auto t1 = std::chrono::steady_clock::now();
  st.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  st.kernel_launches = (int)(h->launches - launches0);
  st.graph_launches = (int)(h->graph_launches - graphs0);
  h->aug_nconv = 0;
  if (stp) *stp = st;
  if (sm_active(h)) PASE_TRY(sm_check_timeout(h));
  PASE_TRY(tc_check(h));
  return rc;
}

int pase_solve_batches(pase_handle h, int nev, int k, int m, double tol, double* lambda, double* U,
                                  pase_stats* stp) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  if (!h->ready) return fail(PASE_ERR_STATE, "pase_setup has not completed");
  if (nev < 1 || k < 1 || m < k + 1 || !(tol > 0.0) || !lambda || !U)
    return fail(PASE_ERR_INVALID_ARG, "pase_solve_batches: bad arguments (need nev >= 1, 1 <= k < m)");
  PASE_TRY(reserve(h, m));
  const int64_t NH = h->NH, N = h->N;
  if (NH < (int64_t)nev + m) return fail(PASE_ERR_INVALID_ARG, "pase_solve_batches: the coarse space needs nev + m pairs");
  if (nev + 3 * m > 1024 && NH + m > 1024)
    return fail(PASE_ERR_INVALID_ARG, "pase_solve_batches: nev + 3m above 1024 pairs of the dense solve");
  PASE_TRY(batch_alloc(h, nev, m));
  auto& b = h->bb;
  Work& w = h->w;
  pase_stats st;
  memset(&st, 0, sizeof(st));
  const int64_t launches0 = h->launches;
  auto t0 = std::chrono::steady_clock::now();
  Stage sg(h);
  void *dl, *dU;
  PASE_TRY(sg.out(lambda, sizeof(double) * nev, &dl));
  PASE_TRY(sg.out(U, sizeof(double) * N * nev, &dU));
  // step 1: the first nev + m coarse pairs (dense)
  DevCSR MHc = h->AH;
  MHc.val = h->MH_val;
  PASE_TRY(launch_csr_to_dense(h, NH, NH, h->AH.rowptr, h->AH.col, h->AH.val, b.AHd, NH));
  PASE_TRY(launch_csr_to_dense(h, NH, NH, MHc.rowptr, MHc.col, MHc.val, b.MHd, NH));
  PASE_TRY(batch_sygv(h, (int)NH, b.top, b.AHd, b.MHd, b.lamH, b.CHc));
  std::vector<double> lamH(b.top), lamw(b.kk), comp(b.nw), lam_out(nev), lam_b(m), rr(m);
  PASE_CUDA(cudaMemcpyAsync(lamH.data(), b.lamH, sizeof(double) * b.top, cudaMemcpyDeviceToHost, h->stream));
  PASE_CUDA(cudaStreamSynchronize(h->stream));
  int rc = PASE_OK;
  double worst_all = 0.0;
  int conv_all = 0;
  // step 2: batches; step 3 for each
  for (const auto& be : batch_bounds(lamH, nev, k)) {
    const int m0 = be.first, kb = be.second - be.first;
    if (kb >= m) {
      rc = fail(PASE_ERR_INVALID_ARG, "pase_solve_batches: a coarse cluster is wider than the block (raise m)");
      break;
    }
    // (a) U = I_H^h u_H[:, m0 .. m0+m), Lambda = lambda_H[m0 .. m0+m)
    PASE_TRY(launch_copy_cols(h, NH, m, b.CHc + m0, b.top, w.CH, m));
    PASE_TRY(launch_csr<double>(h, CSR_MV, m, h->Pd, h->Pd.val, nullptr, w.CH, nullptr, nullptr, nullptr, nullptr, 0.0,
                                w.U, nullptr, nullptr, nullptr));
    for (int j = 0; j < m; ++j) lam_b[j] = lamH[m0 + j];
    PASE_CUDA(cudaMemcpyAsync(w.lam, lam_b.data(), sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
    // (b) the shift: midpoint of the batch's coarse eigenvalues
    const double theta = 0.5 * (lamH[m0] + lamH[m0 + kb - 1]);
    bool conv = false;
    double worst = INFINITY;
    for (int it = 1; it <= h->opt.max_iter && !conv; ++it) {
      st.iterations++;
      // (c) linear solve A_h w = lambda M_h u from u
      PASE_TRY(step_residual(h, w.U, w.lam, w.R));
      PASE_TRY(step_linear_solve(h, w.U, w.W));
      // (d) the pairs of the augmented pencil nearest theta
      PASE_TRY(step_project(h, w.W, w.aH, w.bH, w.GA, w.GM));
      PASE_TRY(batch_assemble(h));
      PASE_TRY(batch_sygv(h, b.n, b.kk, b.Ad, b.Bd, b.lamw, b.Cw));
      PASE_CUDA(cudaMemcpyAsync(lamw.data(), b.lamw, sizeof(double) * b.kk, cudaMemcpyDeviceToHost, h->stream));
      PASE_CUDA(cudaStreamSynchronize(h->stream));
      std::vector<int> order(b.kk);
      for (int i = 0; i < b.kk; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.end(),
                       [&](int a, int c) { return std::fabs(lamw[a] - theta) < std::fabs(lamw[c] - theta); });
      std::vector<int> win(order.begin(), order.begin() + b.nw);
      std::sort(win.begin(), win.end());
      if (win.back() == b.kk - 1 && b.kk < b.n) {
        rc = fail(PASE_ERR_INVALID_ARG, "pase_solve_batches: the window reaches past the computed pairs");
        break;
      }
      // (e) components in span(W): X GM = C_H^T bH + C_W^T GM, ||Pi v_i||_b^2 = X(i,:) GM X(i,:)^T
      PASE_TRY(upload_ints(h, win, b.idx));
      PASE_TRY(launch_gather_cols(h, b.n, b.nw, b.Cw, b.kk, b.idx, b.Cc, b.nw));
      PASE_TRY(ts_gram(h, NH, b.nw, m, b.Cc, b.nw, w.bH, m, b.Rm, m, false));
      PASE_TRY(small_gemm(h, b.nw, m, m, 1.0, b.Cc + NH * b.nw, b.nw, true, w.GM, m, 1.0, b.Rm, m));
      PASE_TRY(launch_transpose(h, b.nw, m, b.Rm, m, b.Rt, b.nw));
      PASE_CUDA(cudaMemcpyAsync(b.Rt2, b.Rt, sizeof(double) * m * b.nw, cudaMemcpyDeviceToDevice, h->stream));
      PASE_TRY(launch_copy_cols(h, m, m, w.GM, m, b.S, m));
      PASE_TRY(small_chol_solve(h, m, b.nw, b.S, m, b.Rt, b.nw, w.status, true));  // X^T = GM^-1 R^T
      PASE_TRY(launch_coldot(h, m, b.nw, b.Rt2, b.Rt, b.comp));
      PASE_CUDA(cudaMemcpyAsync(comp.data(), b.comp, sizeof(double) * b.nw, cudaMemcpyDeviceToHost, h->stream));
      PASE_TRY(sync_small(h, nullptr, 0, w.status, 1));
      if (w.h_status[0] != 0) {
        rc = fail(PASE_ERR_NOT_SPD, "pase_solve_batches: the Gram block of M_h is not positive definite");
        break;
      }
      std::vector<int> pick(b.nw);
      for (int i = 0; i < b.nw; ++i) pick[i] = i;
      std::stable_sort(pick.begin(), pick.end(), [&](int a, int c) { return comp[a] > comp[c]; });
      pick.resize(m);
      std::sort(pick.begin(), pick.end());
      std::vector<int> sel(m);
      for (int j = 0; j < m; ++j) {
        sel[j] = win[pick[j]];
        lam_b[j] = lamw[sel[j]];
      }
      PASE_TRY(upload_ints(h, sel, b.idx));
      PASE_TRY(launch_gather_cols(h, NH, m, b.Cw, b.kk, b.idx, w.CH, m));
      PASE_TRY(launch_gather_cols(h, m, m, b.Cw + NH * b.kk, b.kk, b.idx, w.CW, m));
      PASE_CUDA(cudaMemcpyAsync(w.lam, lam_b.data(), sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
      PASE_TRY(step_prolongate(h, w.W, w.CH, w.CW, w.U));
      // convergence of the owned pairs
      PASE_TRY(step_residual(h, w.U, w.lam, w.R));
      PASE_TRY(sync_small(h, w.relres, m, w.df_flag, w.df_flag ? 1 : 0));
      if (w.df_flag && w.h_status[0]) PASE_TRY(df_check(h));
      worst = 0.0;
      for (int j = 0; j < kb; ++j) worst = std::max(worst, w.h_small[j]);
      if (!(worst == worst)) {
        rc = fail(PASE_ERR_NAN, "pase_solve_batches: NaN in the eigen-residual");
        break;
      }
      if (h->opt.verbose)
        fprintf(stderr, "[pase] batch at %d (%d pairs) iter %d  max relres %.3e\n", m0, kb, it, worst);
      conv = worst <= tol;
      if (!conv) {  // (f) linear solve A_h u = lambda M_h u-hat from u-hat
        PASE_TRY(step_linear_solve(h, w.U, w.W));
        PASE_CUDA(cudaMemcpyAsync(w.U, w.W, sizeof(double) * N * m, cudaMemcpyDeviceToDevice, h->stream));
      }
    }
    if (rc != PASE_OK) break;
    PASE_TRY(launch_copy_cols(h, N, kb, w.U, m, (double*)dU + m0, nev));
    for (int j = 0; j < kb; ++j) lam_out[m0 + j] = lam_b[j];
    worst_all = std::max(worst_all, worst);
    if (conv) conv_all += kb;
    else if (rc == PASE_OK) rc = PASE_ERR_NOT_CONVERGED;
  }
  PASE_CUDA(cudaMemcpyAsync(dl, lam_out.data(), sizeof(double) * nev, cudaMemcpyHostToDevice, h->stream));
  PASE_TRY(sg.finish());
  st.converged = conv_all;
  st.max_residual = worst_all;
  st.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  st.kernel_launches = (int)(h->launches - launches0);
  if (stp) *stp = st;
  if (rc == PASE_ERR_NOT_CONVERGED) set_error("a batch reached the maximum number of iterations");
  PASE_TRY(tc_check(h));
  return rc;
}

// ------------------------------------------------------------------ learned smoother ABI
static void invalidate_graph(pase_ctx* h) {
  if (h->ls_graph) cudaGraphExecDestroy(h->ls_graph);
  h->ls_graph = nullptr;
  h->ls_graph_U = nullptr;
  h->ls_graph_W = nullptr;
  h->ls_last_U = nullptr;
  h->ls_last_W = nullptr;
}

int pase_set_grid(pase_handle h, int dim, int n, const double* log_kappa) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  if (!h->ready) return fail(PASE_ERR_STATE, "pase_set_grid: pase_setup has not completed");
  return sm_set_grid(h, dim, n, log_kappa);
}

int pase_smoother_nparams(int dim) { return smoother_nparams(dim); }

int pase_smoother_state(pase_handle h, float* state, int64_t count, int get) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  PASE_TRY(sm_state(h, state, count, get != 0));
  if (!get) invalidate_graph(h);  // a captured step (a) may hold the Jacobi sweeps
  return PASE_OK;
}

static int ensure_workspace(pase_ctx* h) { return h->w.m == 0 ? reserve(h, 8) : PASE_OK; }

int pase_smoother_apply(pase_handle h, int m, const double* R, double* D) {
  PASE_TRY(check_m(h, m));
  if (!R || !D) return fail(PASE_ERR_INVALID_ARG, "pase_smoother_apply: null argument");
  if (!h->sm || !h->sm->has_params) return fail(PASE_ERR_STATE, "pase_smoother_apply: no grid or parameters");
  Stage st(h);
  const size_t nm = (size_t)h->N * m * sizeof(double);
  const void* dR;
  void* dD;
  PASE_TRY(st.in(R, nm, &dR));
  PASE_TRY(st.out(D, nm, &dD));
  PASE_TRY(sm_apply<double>(h, m, (const double*)dR, m, h->lv[0].dinv, (double*)dD, m, false));
  PASE_TRY(st.finish());
  return sm_check_timeout(h);
}

int pase_smoother_step(pase_handle h, const double* E, const double* R, int update, float lr, float beta1,
                       float beta2, float eps, double* loss8, double* grad) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  if (!E || !R || !loss8) return fail(PASE_ERR_INVALID_ARG, "pase_smoother_step: null argument");
  if (!h->sm || !h->sm->has_params) return fail(PASE_ERR_STATE, "pase_smoother_step: no grid or parameters");
  PASE_TRY(ensure_workspace(h));
  Stage st(h);
  const size_t nb = (size_t)h->N * 8 * sizeof(double);
  const void *dE, *dR;
  PASE_TRY(st.in(E, nb, &dE));
  PASE_TRY(st.in(R, nb, &dR));
  PASE_TRY(sm_step(h, (const double*)dE, (const double*)dR, update != 0, lr, beta1, beta2, eps, loss8));
  if (grad) PASE_TRY(sm_grad_to_host(h, grad));
  if (update) invalidate_graph(h);
  return st.finish();
}

void pase_default_train_options(pase_train_options* o) {
  if (!o) return;
  o->steps = 500;
  o->lr = 1e-3f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->seed = 0;
  o->max_cycles = 2;
}

// Energy-norm error factor ||e0 - x||_A / ||e0||_A (mean over 8 seeded random errors)
// after two V-cycles from zero with the handle's current fine-level smoother.
static int vcycle_energy_factor(pase_ctx* h, unsigned seed, double* factor) {
  Smoother* s = h->sm;
  const int B = 8;
  const int64_t N = h->N;
  const Level& L0 = h->lv[0];
  LevelBufs<double> VB = fp64_bufs(h);
  double* ws = s->sums + 4 * B;  // [2B]: sums e.Ae after and before
  PASE_TRY(launch_hash_fill(h, N, B, B, seed, s->e));
  PASE_TRY(launch_csr<double>(h, CSR_MV, B, L0.A, L0.A.val, nullptr, s->e, nullptr, nullptr, nullptr, nullptr, 0.0,
                              VB.b[0], nullptr, nullptr, nullptr));
  PASE_CUDA(cudaMemsetAsync(VB.x[0], 0, sizeof(double) * N * B, h->stream));
  for (int c = 0; c < 2; ++c) PASE_TRY(vcycle<double>(h, VB, 0, B, c == 0));
  PASE_TRY(launch_coldot(h, N, B, s->e, VB.b[0], ws + B));              // e0 . A e0
  PASE_TRY(launch_axpy(h, N * B, -1.0, VB.x[0], s->e, s->e));          // E = e0 - x
  PASE_TRY(launch_csr<double>(h, CSR_MV, B, L0.A, L0.A.val, nullptr, s->e, nullptr, nullptr, nullptr, nullptr, 0.0,
                              s->r, nullptr, nullptr, nullptr));
  PASE_TRY(launch_coldot(h, N, B, s->e, s->r, ws));                    // E . A E
  PASE_CUDA(cudaMemcpyAsync(s->h_sums, ws, sizeof(double) * 2 * B, cudaMemcpyDeviceToHost, h->stream));
  if (h->stream) PASE_CUDA(cudaStreamSynchronize(h->stream));
  else PASE_CUDA(cudaDeviceSynchronize());
  double f = 0.0;
  for (int b = 0; b < B; ++b) f += sqrt(s->h_sums[b] / s->h_sums[B + b]) / B;
  *factor = f;
  return PASE_OK;
}

int pase_train_smoother(pase_handle h, const pase_train_options* o, double* losses) {
  if (!h || !o || !losses) return fail(PASE_ERR_INVALID_ARG, "pase_train_smoother: null argument");
  if (o->steps < 1 || o->max_cycles < 0 || !(o->lr > 0.f))
    return fail(PASE_ERR_INVALID_ARG, "pase_train_smoother: bad options");
  if (!h->sm || !h->sm->has_params) return fail(PASE_ERR_STATE, "pase_train_smoother: no grid or parameters");
  PASE_TRY(ensure_workspace(h));
  Smoother* s = h->sm;
  const int B = 8;
  const int64_t N = h->N;
  const Level& L0 = h->lv[0];
  const double* dinv = L0.dinv;
  LevelBufs<double> VB = fp64_bufs(h);
  // The samples come from the V-cycle that uses the network being trained (on-policy),
  // so the states it meets after its own sweeps are in the training set.
  struct Restore {
    pase_ctx* h;
    int smoother;
    ~Restore() {
      h->opt.smoother = smoother;
      h->sm_suspend = false;
    }
  } guard{h, h->opt.smoother};
  h->opt.smoother = PASE_SMOOTHER_LEARNED;
  h->sm_suspend = false;
  s->rejected = false;
  invalidate_graph(h);
  auto residual = [&](double* out) {
    return launch_csr<double>(h, CSR_RESID, B, L0.A, L0.A.val, nullptr, VB.x[0], nullptr, VB.b[0], nullptr, nullptr,
                              0.0, out, nullptr, nullptr, nullptr);
  };
  auto sweep = [&](bool from_zero) -> int {  // x <- x + S(b - A x)  (x = S(b) from zero)
    if (from_zero) return sm_apply<double>(h, B, VB.b[0], B, dinv, VB.x[0], B, false);
    PASE_TRY(residual(VB.t1[0]));
    return sm_apply<double>(h, B, VB.t1[0], B, dinv, VB.x[0], B, true);
  };
  const int window = std::min(10, o->steps);
  double first = 0.0, last = 0.0, jac = 0.0, l8[8], j8[8];
  for (int step = 0; step < o->steps; ++step) {
    const unsigned seed = o->seed * 2654435761u + (unsigned)step + 1u;
    PASE_TRY(launch_hash_fill(h, N, B, B, seed, s->e));
    PASE_TRY(launch_csr<double>(h, CSR_MV, B, L0.A, L0.A.val, nullptr, s->e, nullptr, nullptr, nullptr, nullptr, 0.0,
                                VB.b[0], nullptr, nullptr, nullptr));
    PASE_CUDA(cudaMemsetAsync(VB.x[0], 0, sizeof(double) * N * B, h->stream));
    // state: k full V-cycles, then 0: nothing more, 1: one pre-smoothing sweep,
    // 2: all pre-sweeps and the coarse-grid correction, 3: that and one post-sweep
    const int type = step % 4;
    const int k = (step / 4) % (o->max_cycles + 1);
    for (int c = 0; c < k; ++c) PASE_TRY(vcycle<double>(h, VB, 0, B, c == 0));
    if (type >= 1) PASE_TRY(sweep(k == 0));
    if (type >= 2) {
      for (int q = 1; q < h->opt.nu1; ++q) PASE_TRY(sweep(false));
      if (h->L > 1) {
        PASE_TRY(residual(VB.t2[0]));
        PASE_TRY(launch_csr<double>(h, CSR_MV, B, L0.PT, L0.PT.val, nullptr, VB.t2[0], nullptr, nullptr, nullptr,
                                    nullptr, 0.0, VB.b[1], nullptr, nullptr, nullptr));
        PASE_TRY(vcycle<double>(h, VB, 1, B, true));
        PASE_TRY(launch_csr<double>(h, CSR_ADD, B, L0.P, L0.P.val, nullptr, VB.x[1], nullptr, VB.x[0], nullptr,
                                    nullptr, 0.0, VB.x[0], nullptr, nullptr, nullptr));
      }
    }
    if (type == 3) PASE_TRY(sweep(false));
    PASE_TRY(launch_axpy(h, N * B, -1.0, VB.x[0], s->e, s->e));  // e = e0 - x
    PASE_TRY(residual(s->r));
    PASE_TRY(sm_step(h, s->e, s->r, true, o->lr, o->beta1, o->beta2, o->eps, l8));
    double mean = 0.0;
    for (int b = 0; b < B; ++b) mean += l8[b] / B;
    if (!isfinite(mean)) return fail(PASE_ERR_NAN, "pase_train_smoother: loss is not finite");
    if (step < window) first += mean / window;
    if (step >= o->steps - window) {
      last += mean / window;
      PASE_TRY(sm_jacobi_loss(h, s->e, s->r, j8));
      for (int b = 0; b < B; ++b) jac += j8[b] / (B * window);
    }
  }
  // validation on fresh errors: the learned V-cycle must beat the Jacobi V-cycle, else
  // the handle falls back to Jacobi
  double f_learned = 0.0, f_jacobi = 0.0;
  const unsigned vseed = o->seed * 2654435761u + 0x5eed5u;
  PASE_TRY(vcycle_energy_factor(h, vseed, &f_learned));
  h->sm_suspend = true;
  PASE_TRY(vcycle_energy_factor(h, vseed, &f_jacobi));
  h->sm_suspend = false;
  s->rejected = !(f_learned < f_jacobi);
  PASE_TRY(sm_check_timeout(h));
  losses[0] = first;
  losses[1] = last;
  losses[2] = jac;
  losses[3] = f_learned;
  losses[4] = f_jacobi;
  return PASE_OK;
}

int pase_profile_kernel(pase_handle h, int kernel) {
  if (!h) return fail(PASE_ERR_INVALID_ARG, "null handle");
  if (kernel != -1 && kernel != PASE_KERNEL_SPMM_AM_FP64 && kernel != PASE_KERNEL_JACOBI_FP64 &&
      kernel != PASE_KERNEL_JACOBI_FP32)
    return fail(PASE_ERR_INVALID_ARG, "pase_profile_kernel: only the fine-level sparse kernels can be timed live");
  if (h->stream) PASE_CUDA(cudaStreamSynchronize(h->stream));
  h->prof_kernel = kernel;
  h->prof_n = 0;
  return PASE_OK;
}

int pase_profile_read(pase_handle h, int64_t* launches, double* total_ms) {
  if (!h || !launches || !total_ms) return fail(PASE_ERR_INVALID_ARG, "pase_profile_read: bad arguments");
  if (h->stream) PASE_CUDA(cudaStreamSynchronize(h->stream));
  else PASE_CUDA(cudaDeviceSynchronize());
  double sum = 0.0;
  for (size_t i = 0; i < h->prof_n; ++i) {
    float ms = 0.f;
    PASE_CUDA(cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
    sum += ms;
  }
  *launches = (int64_t)h->prof_n;
  *total_ms = sum;
  h->prof_n = 0;
  return PASE_OK;
}

int pase_solve_batched(pase_handle* hs, int count, const int* nev, const double* tol, const int* m,
                       const double* const* U0, double* const* lambda, double* const* U, pase_stats* st) {
  if (count < 0 || (count > 0 && (!hs || !nev || !tol || !lambda || !U)))
    return fail(PASE_ERR_INVALID_ARG, "pase_solve_batched: bad arguments");
  if (count == 0) return PASE_OK;
  if (batch_graph_ok(hs, count)) return solve_batched_graph(hs, count, nev, tol, m, U0, lambda, U, st);
  std::vector<int> rcs(count, PASE_OK);
  std::vector<std::string> msgs(count);
  // Problems whose handles share a CUDA stream run one after another on one thread (a
  // stream cannot be captured and synchronised at once); distinct streams run concurrently.
  // Groups start largest first (work ~ rows x block width) to shorten the tail.
  std::vector<std::vector<int>> groups;
  {
    std::vector<std::pair<cudaStream_t, int>> key;  // stream -> group index
    for (int i = 0; i < count; ++i) {
      const cudaStream_t s = hs[i] ? hs[i]->stream : nullptr;
      int g = -1;
      for (auto& kv : key)
        if (kv.first == s) g = kv.second;
      if (g < 0) {
        g = (int)groups.size();
        key.push_back({s, g});
        groups.emplace_back();
      }
      groups[g].push_back(i);
    }
    auto work = [&](const std::vector<int>& gr) {
      double w = 0.0;
      for (int i : gr) w += hs[i] ? (double)hs[i]->N * (m ? m[i] : nev[i]) : 0.0;
      return w;
    };
    std::stable_sort(groups.begin(), groups.end(),
                     [&](const std::vector<int>& a, const std::vector<int>& b) { return work(a) > work(b); });
  }
  std::atomic<int> next(0);
  const int ngroups = (int)groups.size();
  const int nthreads = std::max(1, std::min(ngroups, 32));
  auto worker = [&]() {
    for (;;) {
      const int g = next.fetch_add(1);
      if (g >= ngroups) break;
      for (int i : groups[g]) {
        if (hs[i]) cudaSetDevice(hs[i]->device);
        pase_stats tmp;
        rcs[i] = pase_solve(hs[i], nev[i], tol[i], m ? m[i] : 0, U0 ? U0[i] : nullptr, lambda[i], U[i],
                            st ? &st[i] : &tmp);
        if (rcs[i] != PASE_OK) msgs[i] = pase_last_error();
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  int rc = PASE_OK;
  for (int i = 0; i < count; ++i)
    if (rcs[i] != PASE_OK && rcs[i] != PASE_ERR_NOT_CONVERGED) {
      return fail(rcs[i], "problem " + std::to_string(i) + ": " + msgs[i]);
    } else if (rcs[i] == PASE_ERR_NOT_CONVERGED) {
      rc = PASE_ERR_NOT_CONVERGED;
    }
  if (rc != PASE_OK) pase::set_error("some problems reached max_iter");
  return rc;
}

}  // extern "C"
