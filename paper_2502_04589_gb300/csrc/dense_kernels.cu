// Dense kernels: tall-skinny Gram products X^T Y and block updates X C over many rows
// (the alpha/beta blocks and the prolongation of Alg. 3 steps 4 and 6, and the block
// operations of the step-(c) eigensolver), the dense coarse-grid multiply, and small
// single-CTA dense routines (symmetric-definite eigensolver, Cholesky solve, GEMM).
//
// FP64 on this part runs at ~1.2 TFLOP/s against ~75 TFLOP/s FP32, so the FP64 kernels
// are ALU-bound: they are laid out to keep the FP64 pipe busy (register tiles fed from
// shared memory) rather than to minimise bytes.
#include <cooperative_groups.h>
#include <float.h>

#include <algorithm>
#include <mutex>

#include "pase_internal.h"

namespace pase {

// ------------------------------------------------------------------ Gram X^T Y
// Thread = one 4x4 tile of G.  blockIdx.y selects a group of 256 tiles, blockIdx.x a
// contiguous row range; rows are staged through shared memory 8 at a time.
// partial[bx][i*k2 + j] receives the block's contribution to G[i][j].
constexpr int kGramRC = 8;

__global__ void __launch_bounds__(256) k_ts_gram(int64_t n, int k1, int k2,
                                                 const double* __restrict__ X, int ldx,
                                                 const double* __restrict__ Y, int ldy, int sym,
                                                 int ntiles, int tiles_j, int64_t rows_per_block,
                                                 double* __restrict__ partial) {
  extern __shared__ double sm[];
  const int k1p = (k1 + 3) & ~3, k2p = (k2 + 3) & ~3;
  double* Xs = sm;                  // [RC][k1p]
  double* Ys = sm + kGramRC * k1p;  // [RC][k2p]
  // tile of this thread
  const int t = blockIdx.y * 256 + threadIdx.x;
  int ti = 0, tj = 0;
  bool have = t < ntiles;
  if (have) {
    if (sym) {
      // enumerate upper tiles (ti <= tj) row by row
      int rem = t, r = 0, len = tiles_j;
      while (rem >= len) {
        rem -= len;
        ++r;
        --len;
      }
      ti = r;
      tj = r + rem;
    } else {
      ti = t / tiles_j;
      tj = t % tiles_j;
    }
  }
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  int64_t r1 = r0 + rows_per_block;
  if (r1 > n) r1 = n;
  for (int64_t rb = r0; rb < r1; rb += kGramRC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kGramRC * k1p; idx += blockDim.x) {
      const int rr = idx / k1p, c = idx % k1p;
      const int64_t row = rb + rr;
      Xs[idx] = (row < r1 && c < k1) ? X[row * ldx + c] : 0.0;
    }
    for (int idx = threadIdx.x; idx < kGramRC * k2p; idx += blockDim.x) {
      const int rr = idx / k2p, c = idx % k2p;
      const int64_t row = rb + rr;
      Ys[idx] = (row < r1 && c < k2) ? Y[row * ldy + c] : 0.0;
    }
    __syncthreads();
    if (have) {
#pragma unroll
      for (int rr = 0; rr < kGramRC; ++rr) {
        double xa[4], yb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xa[a] = Xs[rr * k1p + ti * 4 + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) yb[b] = Ys[rr * k2p + tj * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
      }
    }
  }
  if (have) {
    double* out = partial + (int64_t)blockIdx.x * k1 * k2;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = ti * 4 + a, j = tj * 4 + b;
        if (i < k1 && j < k2) out[i * k2 + j] = acc[a][b];
      }
  }
}

// G[i][j] = sum_b partial[b][i][j]; for sym, lower entries mirror the upper ones.
__global__ void k_gram_reduce(int nb, int k1, int k2, int sym, const double* __restrict__ partial,
                              double* __restrict__ G, int ldg) {
  const int64_t total = (int64_t)k1 * k2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(idx / k2), j = (int)(idx % k2);
    int si = i, sj = j;
    if (sym && i > j) {
      si = j;
      sj = i;
    }
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[(int64_t)b * total + (int64_t)si * k2 + sj];
    G[(int64_t)i * ldg + j] = s;
  }
}

int ts_gram(pase_ctx* h, int64_t n, int k1, int k2, const double* X, int ldx, const double* Y,
            int ldy, double* G, int ldg, bool sym) {
  if (k1 <= 0 || k2 <= 0) return PASE_OK;
  if (sym && k1 != k2) return fail(PASE_ERR_INVALID_ARG, "ts_gram: sym needs k1 == k2");
  const int tiles_i = (k1 + 3) / 4, tiles_j = (k2 + 3) / 4;
  const int ntiles = sym ? tiles_i * (tiles_i + 1) / 2 : tiles_i * tiles_j;
  const int gy = (ntiles + 255) / 256;
  const int64_t budget = (int64_t)(h->w.partial_bytes / sizeof(double));
  int64_t gx = 608 / gy;
  if (gx < 1) gx = 1;
  const int64_t max_by_rows = (n + 63) / 64;
  if (gx > max_by_rows) gx = max_by_rows;
  if (gx * k1 * k2 > budget) gx = budget / ((int64_t)k1 * k2);
  if (gx < 1) return fail(PASE_ERR_INVALID_ARG, "ts_gram: partial buffer too small");
  int64_t rpb = (n + gx - 1) / gx;
  rpb = (rpb + kGramRC - 1) / kGramRC * kGramRC;
  gx = (n + rpb - 1) / rpb;
  if (gx < 1) gx = 1;
  const size_t smem = (size_t)kGramRC * (((k1 + 3) & ~3) + ((k2 + 3) & ~3)) * sizeof(double);
  PASE_TRY(ensure_max_smem((const void*)k_ts_gram, 200 * 1024));
  dim3 grid((unsigned)gx, (unsigned)gy);
  k_ts_gram<<<grid, 256, smem, h->stream>>>(n, k1, k2, X, ldx, Y, ldy, sym ? 1 : 0, ntiles, tiles_j,
                                            rpb, h->w.partial);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  const int64_t total = (int64_t)k1 * k2;
  int rg = (int)((total + 255) / 256);
  k_gram_reduce<<<rg, 256, 0, h->stream>>>((int)gx, k1, k2, sym ? 1 : 0, h->w.partial, G, ldg);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// ------------------------------------------------------------------ Y = a X C + b Y
// Thread group of tpr = ceil(k2/2) threads per row, 2 output columns each; C staged in
// shared memory 32 rows at a time.
template <typename T>
__global__ void __launch_bounds__(256) k_ts_gemm(int64_t n, int k1, int k2, T alpha,
                                                 const T* __restrict__ X, int64_t ldx,
                                                 const T* __restrict__ C, int ldc, T beta,
                                                 T* __restrict__ Y, int64_t ldy, int tpr, int rpb) {
  extern __shared__ unsigned char smraw[];
  T* Cs = reinterpret_cast<T*>(smraw);  // [32][k2p]
  const int k2p = tpr * 2;
  const int tx = threadIdx.x % tpr, ty = threadIdx.x / tpr;
  const int64_t row = (int64_t)blockIdx.x * rpb + ty;
  const bool active = ty < rpb && row < n;
  const int c0 = tx * 2;
  T acc0 = 0, acc1 = 0;
  for (int kb = 0; kb < k1; kb += 32) {
    const int kc = min(32, k1 - kb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * k2p; idx += blockDim.x) {
      const int r = idx / k2p, c = idx % k2p;
      Cs[idx] = (r < kc && c < k2) ? C[(int64_t)(kb + r) * ldc + c] : T(0);
    }
    __syncthreads();
    if (active) {
      const T* xr = X + row * ldx + kb;
      for (int r = 0; r < kc; ++r) {
        const T x = xr[r];
        acc0 = fma(x, Cs[r * k2p + c0], acc0);
        acc1 = fma(x, Cs[r * k2p + c0 + 1], acc1);
      }
    }
  }
  if (active) {
    T* yr = Y + row * ldy;
    if (c0 < k2) yr[c0] = (beta == T(0)) ? alpha * acc0 : fma(alpha, acc0, beta * yr[c0]);
    if (c0 + 1 < k2) yr[c0 + 1] = (beta == T(0)) ? alpha * acc1 : fma(alpha, acc1, beta * yr[c0 + 1]);
  }
}

template <typename T>
static int ts_gemm_t(pase_ctx* h, int64_t n, int k1, int k2, double alpha, const T* X, int64_t ldx,
                     const T* C, int ldc, double beta, T* Y, int64_t ldy) {
  if (n == 0 || k2 == 0) return PASE_OK;
  const int tpr = (k2 + 1) / 2;
  if (tpr > 256) return fail(PASE_ERR_INVALID_ARG, "ts_gemm: k2 too large");
  const int rpb = 256 / tpr;
  const int64_t grid = (n + rpb - 1) / rpb;
  const size_t smem = (size_t)32 * tpr * 2 * sizeof(T);
  PASE_TRY(ensure_max_smem((const void*)k_ts_gemm<T>, 200 * 1024));
  k_ts_gemm<T><<<(unsigned)grid, 256, smem, h->stream>>>(n, k1, k2, (T)alpha, X, ldx, C, ldc, (T)beta,
                                                         Y, ldy, tpr, rpb);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

int ts_gemm(pase_ctx* h, int64_t n, int k1, int k2, double alpha, const double* X, int ldx,
            const double* C, int ldc, double beta, double* Y, int ldy) {
  return ts_gemm_t<double>(h, n, k1, k2, alpha, X, ldx, C, ldc, beta, Y, ldy);
}

template <typename T>
int dense_mm(pase_ctx* h, int64_t n, int m, const T* Ainv, const T* B, T* X) {
  return ts_gemm_t<T>(h, n, (int)n, m, 1.0, Ainv, n, B, m, 0.0, X, m);
}
template int dense_mm<double>(pase_ctx*, int64_t, int, const double*, const double*, double*);
template int dense_mm<float>(pase_ctx*, int64_t, int, const float*, const float*, float*);

// ------------------------------------------------------------------ small GEMM
// C[i][j] = alpha sum_l op(A)[i][l] B[l][j] + beta C[i][j]; op(A) = A or A^T.
__global__ void k_small_gemm(int m, int n, int k, double alpha, const double* __restrict__ A,
                             int lda, int transA, const double* __restrict__ B, int ldb,
                             double beta, double* __restrict__ C, int ldc) {
  const int64_t total = (int64_t)m * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    double s = 0.0;
    if (transA)
      for (int l = 0; l < k; ++l) s = fma(A[(int64_t)l * lda + i], B[(int64_t)l * ldb + j], s);
    else
      for (int l = 0; l < k; ++l) s = fma(A[(int64_t)i * lda + l], B[(int64_t)l * ldb + j], s);
    C[(int64_t)i * ldc + j] = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * C[(int64_t)i * ldc + j]);
  }
}
int small_gemm(pase_ctx* h, int m, int n, int k, double alpha, const double* A, int lda,
               bool transA, const double* B, int ldb, double beta, double* C, int ldc) {
  const int64_t total = (int64_t)m * n;
  if (total == 0) return PASE_OK;
  int g = (int)((total + 127) / 128);
  if (g > 152 * 8) g = 152 * 8;
  k_small_gemm<<<g, 128, 0, h->stream>>>(m, n, k, alpha, A, lda, transA ? 1 : 0, B, ldb, beta, C, ldc);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// ------------------------------------------------------------------ block reductions
__device__ double block_sum(double v, double* red) {
  // red: >= 33 doubles of shared memory; warp partials, then a shuffle tree in warp 0
  // (a serial FP64 sum would be a long dependent chain on this part)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// ------------------------------------------------------------------ small Cholesky solve
// One CTA: S (n x n, lower used) <- its Cholesky factor L, then B (n x nrhs) <- S^-1 B.
// status[0] = 1 if a pivot is not positive.
__global__ void __launch_bounds__(1024) k_small_chol_solve(int n, int nrhs, double* S, int lds,
                                                           double* B, int ldb, int* status,
                                                           int factor) {
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; factor && j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = S[(int64_t)j * lds + j];
      if (!(d > 0.0) || !isfinite(d)) s_fail = 1;
      else S[(int64_t)j * lds + j] = sqrt(d);
    }
    __syncthreads();
    if (s_fail) break;
    const double ljj = S[(int64_t)j * lds + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) S[(int64_t)i * lds + j] /= ljj;
    __syncthreads();
    const int len = n - j - 1;
    for (int idx = threadIdx.x; idx < len * len; idx += blockDim.x) {
      const int i = j + 1 + idx / len, l = j + 1 + idx % len;
      if (l <= i) S[(int64_t)i * lds + l] -= S[(int64_t)i * lds + j] * S[(int64_t)l * lds + j];
    }
    __syncthreads();
  }
  if (s_fail) {
    if (threadIdx.x == 0) status[0] = 1;
    return;
  }
  // forward: L y = b ; backward: L^T x = y  (parallel over right-hand sides)
  for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      double s = B[(int64_t)i * ldb + c];
      for (int l = 0; l < i; ++l) s -= S[(int64_t)i * lds + l] * B[(int64_t)l * ldb + c];
      B[(int64_t)i * ldb + c] = s / S[(int64_t)i * lds + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = B[(int64_t)i * ldb + c];
      for (int l = i + 1; l < n; ++l) s -= S[(int64_t)l * lds + i] * B[(int64_t)l * ldb + c];
      B[(int64_t)i * ldb + c] = s / S[(int64_t)i * lds + i];
    }
  }
}
int small_chol_solve(pase_ctx* h, int n, int nrhs, double* S, int lds, double* B, int ldb,
                     int* status_dev, bool factor) {
  k_small_chol_solve<<<1, 1024, 0, h->stream>>>(n, nrhs, S, lds, B, ldb, status_dev, factor ? 1 : 0);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// ------------------------------------------------------------------ small eigensolver
// The k smallest pairs of GA c = lambda GB c (n x n symmetric, GB positive semi-definite),
// FP64, as five kernels so that only the inherently sequential parts run on one SM (FP64
// issues at ~2 FMA/clock per SM on this part, so work spread over many SMs matters):
//  1. (1 CTA)   scaling D = diag(GB)^-1/2 and Cholesky D GB D = L L^T with dropping of
//               numerically dependent directions (scaled pivot below kPivTol; a zero
//               diagonal, i.e. a locked search direction, is dropped too);
//  2. (n CTAs)  K = L^-1 (D GA D) L^-T by two column-parallel forward substitutions;
//  3. (1 CTA)   Householder tridiagonalisation Q^T K Q = T, then the k smallest
//               eigenvalues of T located by multisection on FP32 Sturm counts;
//  4. (k CTAs)  eigenvectors of T by inverse iteration with Rayleigh-quotient shifts (FP64
//               accuracy); close eigenvalues form a cluster, re-orthogonalised and rotated
//               by a Rayleigh-Ritz step inside the cluster; lam[i] = Rayleigh quotient;
//  5. (k/4 CTAs) back-transform c = D L^-T Q z.
// Output C (n x k, ldc) is GB-orthonormal.  Dropped directions get an eigenvalue above the
// kept spectrum; status[0] = 1 only if fewer than k directions remain (or GB is invalid).
constexpr double kPivTol = 1e-10;
constexpr int kClusterRR = 16;

struct SygvWork {
  double *K, *L, *Y, *Z, *d, *e, *tau, *sc, *lamx;
  int* info;  // [0] dropped count, [1] cluster flag scratch
};
__device__ __host__ inline SygvWork sygv_work(double* w, int n, int k) {
  SygvWork s;
  s.K = w;
  s.L = s.K + (size_t)n * n;
  s.Y = s.L + (size_t)n * n;
  s.Z = s.Y + (size_t)n * n;
  s.d = s.Z + (size_t)n * k;
  s.e = s.d + n;
  s.tau = s.e + n;  // drop mask (1 = dropped) in kernels 1-2, reflector taus after kernel 3
  s.sc = s.tau + n;
  s.lamx = s.sc + n;
  s.info = reinterpret_cast<int*>(s.lamx + k + 1);
  return s;
}

__device__ int sturm_count_f32(int n, const float* d, const float* e2, float x) {
  // FP32 count of eigenvalues below x (used only to locate eigenvalues to ~1e-6 |T|)
  int cnt = 0;
  float q = d[0] - x;
  if (q < 0.f) ++cnt;
  for (int i = 1; i < n; ++i) {
    if (q == 0.f) q = -1e-30f;
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (q < 0.f) ++cnt;
  }
  return cnt;
}

__device__ double hash_unit(unsigned a, unsigned b) {
  unsigned long long z = ((unsigned long long)a << 32) ^ b ^ 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// 1/x: FP32 seed refined by two FP64 Newton steps (a much shorter dependent chain than
// FP64 division on this part; accurate to about one ulp), true division outside FP32 range.
__device__ __forceinline__ double fast_rcp(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
  double r = (double)(1.0f / (float)x);
  r = r * fma(-x, r, 2.0);
  r = r * fma(-x, r, 2.0);
  return r;
}

// Solve (T - lam I) x = b in place (b -> x), tridiagonal LU with partial pivoting.
__device__ void tri_solve(int n, const double* d, const double* e, double lam, double* b,
                          double* u0, double* u1, double* u2, double tiny) {
  for (int i = 0; i < n; ++i) {
    u0[i] = d[i] - lam;
    u1[i] = (i < n - 1) ? e[i] : 0.0;
    u2[i] = 0.0;
  }
  for (int i = 0; i < n - 1; ++i) {
    const double sub = e[i];  // element (i+1, i)
    if (fabs(u0[i]) >= fabs(sub)) {
      if (u0[i] == 0.0) u0[i] = tiny;
      const double f = sub * fast_rcp(u0[i]);
      u0[i + 1] -= f * u1[i];
      b[i + 1] -= f * b[i];
    } else {
      const double f = u0[i] * fast_rcp(sub);
      const double r1 = u0[i + 1], r2 = (i + 1 < n - 1) ? e[i + 1] : 0.0;
      const double o1 = u1[i];
      u0[i] = sub;
      u1[i] = r1;
      u2[i] = r2;
      u0[i + 1] = o1 - f * r1;
      if (i + 1 < n - 1) u1[i + 1] = -f * r2;
      const double bi = b[i];
      b[i] = b[i + 1];
      b[i + 1] = bi - f * b[i + 1];
    }
  }
  if (u0[n - 1] == 0.0) u0[n - 1] = tiny;
  b[n - 1] *= fast_rcp(u0[n - 1]);
  if (n >= 2) {
    b[n - 2] = (b[n - 2] - u1[n - 2] * b[n - 1]) * fast_rcp(u0[n - 2]);
    for (int i = n - 3; i >= 0; --i) b[i] = (b[i] - u1[i] * b[i + 1] - u2[i] * b[i + 2]) * fast_rcp(u0[i]);
  }
}

// 1. scaling + Cholesky with dropping (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024) k_sygv_chol(int n, int k, const double* __restrict__ GA, int lda,
                                                    const double* __restrict__ GB, int ldb, double* work,
                                                    int* status) {
  __shared__ int s_fail, s_drop;
  extern __shared__ double colj[];  // n
  SygvWork W = sygv_work(work, n, k);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  if (tid == 0) {
    s_fail = 0;
    s_drop = 0;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const double g = GB[(int64_t)i * ldb + i];
    if (!(g >= 0.0) || !isfinite(g)) s_fail = 1;
    W.sc[i] = (g > 0.0) ? rsqrt(g) : 0.0;
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) status[0] = 1;
    return;
  }
  for (int i = warp; i < n; i += nwarps)
    for (int j = lane; j < n; j += 32) {
      const double s = W.sc[i] * W.sc[j];
      W.K[(int64_t)i * n + j] = s * 0.5 * (GA[(int64_t)i * lda + j] + GA[(int64_t)j * lda + i]);
      W.L[(int64_t)i * n + j] = s * 0.5 * (GB[(int64_t)i * ldb + j] + GB[(int64_t)j * ldb + i]);
    }
  __syncthreads();
  __shared__ double s_inv;
  __shared__ int s_dropj;
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {  // pivot, its square root and reciprocal once (FP64 sqrt/div are costly)
      const double dj = W.L[(int64_t)j * n + j];
      const bool drop = !(dj > kPivTol) || !isfinite(dj);
      const double ljj = drop ? 1.0 : sqrt(dj);
      s_inv = drop ? 0.0 : 1.0 / ljj;
      s_dropj = drop ? 1 : 0;
      W.L[(int64_t)j * n + j] = ljj;
      W.tau[j] = drop ? 1.0 : 0.0;
      if (drop) ++s_drop;
    }
    __syncthreads();
    const bool drop = s_dropj != 0;
    const double inv = s_inv;
    const int len = n - j - 1;
    for (int r = tid; r < len; r += nt) colj[r] = W.L[(int64_t)(j + 1 + r) * n + j] * inv;
    __syncthreads();
    for (int r = tid; r < len; r += nt) W.L[(int64_t)(j + 1 + r) * n + j] = colj[r];
    if (!drop)
      for (int r = warp; r < len; r += nwarps) {
        double* Lr = W.L + (int64_t)(j + 1 + r) * n + (j + 1);
        const double cr = colj[r];
        for (int c = lane; c <= r; c += 32) Lr[c] -= cr * colj[c];
      }
    __syncthreads();
  }
  for (int i = warp; i < n; i += nwarps)
    for (int j = i + 1 + lane; j < n; j += 32) W.L[(int64_t)i * n + j] = 0.0;
  if (tid == 0) {
    W.info[0] = s_drop;
    status[0] = (n - s_drop < k) ? 1 : 0;
  }
}

// 2. out[c-th vector] = L^-1 in[c-th vector], one CTA per vector.  pass 0: input row c of
//    K (= column c, K symmetric), output column c of Y; pass 1: input row c of Y, output
//    row c of K (K <- L^-1 K L^-T since K' = (L^-1 Y^T)^T and K' is symmetric).
__global__ void __launch_bounds__(128) k_sygv_trsm(int n, int k, double* work, int pass, int stage_l, int cpc,
                                                   const int* status) {
  // the four warps stage the right-hand sides, the reciprocal pivots and (stage_l) the
  // packed L in shared memory; warps 0..cpc-1 then each run one column's n dependent
  // substitution steps with shuffles only (no block barrier in the loop).  cpc columns per
  // CTA keep the grid within one wave of the SMs.
  if (status[0] != 0) return;
  extern __shared__ double sy[];  // per column: n solution and n right-hand side entries; n reciprocal pivots; [packed L]
  double* rinv = sy + (size_t)2 * cpc * n;
  double* Lp = rinv + n;          // row i of L at Lp + i(i+1)/2 when staged
  SygvWork W = sygv_work(work, n, k);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = blockIdx.x * cpc;
  for (int q = 0; q < cpc && c0 + q < n; ++q) {
    const double* in = (pass == 0) ? W.K + (int64_t)(c0 + q) * n : W.Y + (int64_t)(c0 + q) * n;
    for (int i = tid; i < n; i += blockDim.x) sy[(size_t)(2 * q + 1) * n + i] = in[i];
  }
  for (int i = tid; i < n; i += blockDim.x) rinv[i] = 1.0 / W.L[(int64_t)i * n + i];
  if (stage_l)
    for (int i = warp; i < n; i += (int)(blockDim.x >> 5))
      for (int l = lane; l <= i; l += 32) Lp[i * (i + 1) / 2 + l] = W.L[(int64_t)i * n + l];
  __syncthreads();
  const int c = c0 + warp;
  if (warp >= cpc || c >= n) return;
  double* x = sy + (size_t)2 * warp * n;
  double* rhs = x + n;
  // column-oriented substitution: lane r % 32 owns row r of the right-hand side; step i
  // computes x_i on its owner lane, broadcasts it, and every lane takes L[r][i] x_i off
  // its rows r > i, so the dependent chain of a step is one multiply, one shuffle and one
  // FMA (no reduction)
  for (int i = 0; i < n; ++i) {
    const double xi = __shfl_sync(0xffffffffu, rhs[i] * rinv[i], i & 31);
    if (lane == (i & 31)) x[i] = xi;
    for (int r = i + 1 + ((lane - (i + 1)) & 31); r < n; r += 32) {
      const double lri = stage_l ? Lp[r * (r + 1) / 2 + i] : W.L[(int64_t)r * n + i];
      rhs[r] = fma(-lri, xi, rhs[r]);
    }
  }
  __syncwarp();
  if (pass == 0)
    for (int i = lane; i < n; i += 32) W.Y[(int64_t)i * n + c] = x[i];
  else
    for (int i = lane; i < n; i += 32) W.K[(int64_t)c * n + i] = x[i];
}

// 3. Householder tridiagonalisation and FP32 multisection (one CTA of 1024 threads).
//    Reflector j acts on rows/cols j+1..n-1; its vector (v[0] = 1 implicit) is kept in
//    row j, K[j][j+2..n-1], and tau[j].
__global__ void __launch_bounds__(1024) k_sygv_tridiag(int n, int k, double* work, const int* status) {
  if (status[0] != 0) return;
  extern __shared__ double shm[];
  __shared__ double red[40];
  __shared__ double s_lo, s_hi, s_hh[3];
  SygvWork W = sygv_work(work, n, k);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  double* v = shm;        // n
  double* p = v + n;      // n
  double* part = p + n;   // nt
  int* icnt = reinterpret_cast<int*>(part + nt);  // nt
  float* df = reinterpret_cast<float*>(icnt + nt);
  float* e2f = df + n;
  float* flo = e2f + n;
  float* fhi = flo + k;
  double* K = W.K;
  // symmetrise; dropped directions get an eigenvalue just above the kept spectrum
  for (int i = warp; i < n; i += nwarps)
    for (int j = i + 1 + lane; j < n; j += 32) {
      const double a = 0.5 * (K[(int64_t)i * n + j] + K[(int64_t)j * n + i]);
      K[(int64_t)i * n + j] = a;
      K[(int64_t)j * n + i] = a;
    }
  __syncthreads();
  if (W.info[0] > 0) {
    double rmax = 0.0;
    for (int i = tid; i < n; i += nt) {
      if (W.tau[i] != 0.0) continue;
      double r = 0.0;
      for (int j = 0; j < n; ++j)
        if (W.tau[j] == 0.0) r += fabs(K[(int64_t)i * n + j]);
      rmax = fmax(rmax, r);
    }
    const double big = 2.0 * block_max(rmax, red) + 1.0;
    for (int i = warp; i < n; i += nwarps)
      for (int j = lane; j < n; j += 32)
        if (W.tau[i] != 0.0 || W.tau[j] != 0.0) K[(int64_t)i * n + j] = (i == j) ? big : 0.0;
    __syncthreads();
  }
  for (int j = 0; j + 2 < n; ++j) {
    const int len = n - j - 1;
    const double* xr = K + (int64_t)j * n + (j + 1);  // row j = column j (symmetric)
    double* A22 = K + (int64_t)(j + 1) * n + (j + 1);
    double part_s = 0.0;
    for (int r = 1 + tid; r < len; r += nt) part_s += xr[r] * xr[r];
    const double sig = block_sum(part_s, red);
    if (tid == 0) {  // reflector scalars once (FP64 sqrt/div are costly), broadcast below
      const double x0 = xr[0];
      double beta = x0, t = 0.0, scal = 0.0;
      if (sig != 0.0) {
        const double nrm = sqrt(x0 * x0 + sig);
        beta = (x0 >= 0.0) ? -nrm : nrm;
        t = (beta - x0) / beta;
        scal = 1.0 / (x0 - beta);
      }
      s_hh[0] = beta;
      s_hh[1] = t;
      s_hh[2] = scal;
    }
    __syncthreads();
    const double beta = s_hh[0], t = s_hh[1], scal = s_hh[2];
    for (int r = tid; r < len; r += nt) v[r] = (r == 0) ? 1.0 : xr[r] * scal;
    __syncthreads();
    if (t != 0.0) {
      for (int r = warp; r < len; r += nwarps) {  // p = t A22 v, one warp per row
        const double* row = A22 + (int64_t)r * n;
        double acc = 0.0;
        for (int c = lane; c < len; c += 32) acc = fma(row[c], v[c], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) p[r] = t * acc;
      }
      __syncthreads();
      double pv = 0.0;
      for (int r = tid; r < len; r += nt) pv += p[r] * v[r];
      const double Kc = 0.5 * t * block_sum(pv, red);
      for (int r = tid; r < len; r += nt) p[r] -= Kc * v[r];
      __syncthreads();
      for (int r = warp; r < len; r += nwarps) {
        double* row = A22 + (int64_t)r * n;
        const double vr = v[r], pr = p[r];
        for (int c = lane; c < len; c += 32) row[c] -= vr * p[c] + pr * v[c];
      }
    }
    __syncthreads();
    if (tid == 0) {
      W.d[j] = K[(int64_t)j * n + j];
      W.e[j] = beta;
      W.tau[j] = t;
    }
    for (int r = 1 + tid; r < len; r += nt) K[(int64_t)j * n + (j + 1 + r)] = v[r];
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      W.d[n - 2] = K[(int64_t)(n - 2) * n + (n - 2)];
      W.e[n - 2] = K[(int64_t)(n - 1) * n + (n - 2)];
      W.tau[n - 2] = 0.0;
    }
    W.d[n - 1] = K[(int64_t)(n - 1) * n + (n - 1)];
    W.e[n - 1] = 0.0;
    W.tau[n - 1] = 0.0;
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(W.e[i - 1]) : 0.0) + (i < n - 1 ? fabs(W.e[i]) : 0.0);
      lo = fmin(lo, W.d[i] - r);
      hi = fmax(hi, W.d[i] + r);
    }
    s_lo = lo;
    s_hi = hi;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    df[i] = (float)W.d[i];
    e2f[i] = (float)(W.e[i] * W.e[i]);
  }
  for (int i = tid; i < k; i += nt) {
    flo[i] = (float)s_lo - 1e-6f * (float)fabs(s_lo) - 1e-30f;
    fhi[i] = (float)s_hi + 1e-6f * (float)fabs(s_hi) + 1e-30f;
  }
  __syncthreads();
  const int G = max(1, min(32, nt / k));
  for (int round = 0; round < 40; ++round) {
    const int i = tid / G, g = tid % G;
    if (i < k) {
      const float a = flo[i], b = fhi[i];
      const float x = a + (b - a) * (float)(g + 1) / (float)(G + 1);
      icnt[tid] = (b - a > 4e-7f * fmaxf(fabsf(a), fabsf(b)) + 1e-30f) ? sturm_count_f32(n, df, e2f, x) : -1;
    }
    __syncthreads();
    int moved = 0;
    if (i < k && g == 0 && icnt[tid] >= 0) {
      const float a = flo[i], b = fhi[i];
      float na = a, nb = b;
      for (int q = 0; q < G; ++q) {
        const float x = a + (b - a) * (float)(q + 1) / (float)(G + 1);
        if (icnt[i * G + q] > i) {
          nb = x;
          break;
        }
        na = x;
      }
      flo[i] = na;
      fhi[i] = nb;
      moved = 1;
    }
    if (block_sum((double)moved, red) == 0.0) break;
  }
  for (int i = tid; i < k; i += nt) W.lamx[i] = 0.5 * ((double)flo[i] + (double)fhi[i]);
  if (tid == 0) W.lamx[k] = fmax(fabs(s_lo), fabs(s_hi));  // |T| bound
}

// Shared-memory variants of kernels 1 and 3 for n(n+1)/2 doubles that fit in shared memory:
// the lower triangle is kept packed (row r at r(r+1)/2), so every access in the long
// sequential loops is a shared-memory access and the rank-2 update touches half the matrix.
__device__ __forceinline__ int tri_idx(int r, int c) { return r * (r + 1) / 2 + c; }  // c <= r

__global__ void __launch_bounds__(1024) k_sygv_chol_s(int n, int k, const double* __restrict__ GA, int lda,
                                                      const double* __restrict__ GB, int ldb, double* work,
                                                      int* status) {
  __shared__ int s_fail, s_drop, s_dropj;
  __shared__ double s_inv;
  extern __shared__ double sm_c[];
  double* Lp = sm_c;                   // n(n+1)/2
  double* colj = Lp + n * (n + 1) / 2; // n
  SygvWork W = sygv_work(work, n, k);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  if (tid == 0) {
    s_fail = 0;
    s_drop = 0;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const double g = GB[(int64_t)i * ldb + i];
    if (!(g >= 0.0) || !isfinite(g)) s_fail = 1;
    W.sc[i] = (g > 0.0) ? rsqrt(g) : 0.0;
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) status[0] = 1;
    return;
  }
  for (int i = warp; i < n; i += nwarps)
    for (int j = lane; j < n; j += 32) {
      const double s = W.sc[i] * W.sc[j];
      W.K[(int64_t)i * n + j] = s * 0.5 * (GA[(int64_t)i * lda + j] + GA[(int64_t)j * lda + i]);
      if (j <= i) Lp[tri_idx(i, j)] = s * 0.5 * (GB[(int64_t)i * ldb + j] + GB[(int64_t)j * ldb + i]);
    }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double dj = Lp[tri_idx(j, j)];
      const bool drop = !(dj > kPivTol) || !isfinite(dj);
      const double ljj = drop ? 1.0 : sqrt(dj);
      s_inv = drop ? 0.0 : 1.0 / ljj;
      s_dropj = drop ? 1 : 0;
      Lp[tri_idx(j, j)] = ljj;
      W.tau[j] = drop ? 1.0 : 0.0;
      if (drop) ++s_drop;
    }
    __syncthreads();
    const bool drop = s_dropj != 0;
    const double inv = s_inv;
    const int len = n - j - 1;
    for (int r = tid; r < len; r += nt) {
      const double x = Lp[tri_idx(j + 1 + r, j)] * inv;
      Lp[tri_idx(j + 1 + r, j)] = x;
      colj[r] = x;
    }
    __syncthreads();
    if (!drop)
      for (int r = warp; r < len; r += nwarps) {
        double* Lr = Lp + tri_idx(j + 1 + r, j + 1);
        const double cr = colj[r];
        for (int c = lane; c <= r; c += 32) Lr[c] -= cr * colj[c];
      }
    __syncthreads();
  }
  for (int i = warp; i < n; i += nwarps)
    for (int j = lane; j < n; j += 32) W.L[(int64_t)i * n + j] = (j <= i) ? Lp[tri_idx(i, j)] : 0.0;
  if (tid == 0) {
    W.info[0] = s_drop;
    status[0] = (n - s_drop < k) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(1024) k_sygv_tridiag_s(int n, int k, double* work, const int* status) {
  if (status[0] != 0) return;
  extern __shared__ double sm_t[];
  __shared__ double red[40];
  __shared__ double s_lo, s_hi, s_hh[3];
  SygvWork W = sygv_work(work, n, k);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  double* Ap = sm_t;                     // n(n+1)/2, packed lower triangle
  double* v = Ap + n * (n + 1) / 2;      // n
  double* p = v + n;                     // n
  int* icnt = reinterpret_cast<int*>(p + n);  // nt
  float* df = reinterpret_cast<float*>(icnt + nt);
  float* e2f = df + n;
  float* flo = e2f + n;
  float* fhi = flo + k;
  const double* K = W.K;
  for (int i = warp; i < n; i += nwarps)
    for (int j = lane; j <= i; j += 32) Ap[tri_idx(i, j)] = 0.5 * (K[(int64_t)i * n + j] + K[(int64_t)j * n + i]);
  __syncthreads();
  if (W.info[0] > 0) {
    double rmax = 0.0;
    for (int i = tid; i < n; i += nt) {
      if (W.tau[i] != 0.0) continue;
      double r = 0.0;
      for (int j = 0; j < n; ++j)
        if (W.tau[j] == 0.0) r += fabs(j <= i ? Ap[tri_idx(i, j)] : Ap[tri_idx(j, i)]);
      rmax = fmax(rmax, r);
    }
    const double big = 2.0 * block_max(rmax, red) + 1.0;
    for (int i = warp; i < n; i += nwarps)
      for (int j = lane; j <= i; j += 32)
        if (W.tau[i] != 0.0 || W.tau[j] != 0.0) Ap[tri_idx(i, j)] = (i == j) ? big : 0.0;
    __syncthreads();
  }
  for (int j = 0; j + 2 < n; ++j) {
    const int len = n - j - 1, j1 = j + 1;
    double part_s = 0.0;
    for (int r = 1 + tid; r < len; r += nt) {
      const double x = Ap[tri_idx(j1 + r, j)];
      part_s += x * x;
    }
    const double sig = block_sum(part_s, red);
    if (tid == 0) {
      const double x0 = Ap[tri_idx(j1, j)];
      double beta = x0, t = 0.0, scal = 0.0;
      if (sig != 0.0) {
        const double nrm = sqrt(x0 * x0 + sig);
        beta = (x0 >= 0.0) ? -nrm : nrm;
        t = (beta - x0) / beta;
        scal = 1.0 / (x0 - beta);
      }
      s_hh[0] = beta;
      s_hh[1] = t;
      s_hh[2] = scal;
    }
    __syncthreads();
    const double beta = s_hh[0], t = s_hh[1], scal = s_hh[2];
    for (int r = tid; r < len; r += nt) v[r] = (r == 0) ? 1.0 : Ap[tri_idx(j1 + r, j)] * scal;
    __syncthreads();
    if (t != 0.0) {
      for (int r = warp; r < len; r += nwarps) {  // p = t A22 v, A22 symmetric from the packed triangle
        const int R = j1 + r;
        double acc = 0.0;
        for (int c = lane; c < len; c += 32) {
          const int C = j1 + c;
          acc = fma(c <= r ? Ap[tri_idx(R, C)] : Ap[tri_idx(C, R)], v[c], acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) p[r] = t * acc;
      }
      __syncthreads();
      double pv = 0.0;
      for (int r = tid; r < len; r += nt) pv += p[r] * v[r];
      const double Kc = 0.5 * t * block_sum(pv, red);
      for (int r = tid; r < len; r += nt) p[r] -= Kc * v[r];
      __syncthreads();
      for (int r = warp; r < len; r += nwarps) {  // lower triangle only
        double* row = Ap + tri_idx(j1 + r, j1);
        const double vr = v[r], pr = p[r];
        for (int c = lane; c <= r; c += 32) row[c] -= vr * p[c] + pr * v[c];
      }
    }
    __syncthreads();
    if (tid == 0) {
      W.d[j] = Ap[tri_idx(j, j)];
      W.e[j] = beta;
      W.tau[j] = t;
    }
    for (int r = 1 + tid; r < len; r += nt) W.K[(int64_t)j * n + (j1 + r)] = v[r];  // reflector store
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      W.d[n - 2] = Ap[tri_idx(n - 2, n - 2)];
      W.e[n - 2] = Ap[tri_idx(n - 1, n - 2)];
      W.tau[n - 2] = 0.0;
    }
    W.d[n - 1] = Ap[tri_idx(n - 1, n - 1)];
    W.e[n - 1] = 0.0;
    W.tau[n - 1] = 0.0;
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(W.e[i - 1]) : 0.0) + (i < n - 1 ? fabs(W.e[i]) : 0.0);
      lo = fmin(lo, W.d[i] - r);
      hi = fmax(hi, W.d[i] + r);
    }
    s_lo = lo;
    s_hi = hi;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    df[i] = (float)W.d[i];
    e2f[i] = (float)(W.e[i] * W.e[i]);
  }
  for (int i = tid; i < k; i += nt) {
    flo[i] = (float)s_lo - 1e-6f * (float)fabs(s_lo) - 1e-30f;
    fhi[i] = (float)s_hi + 1e-6f * (float)fabs(s_hi) + 1e-30f;
  }
  __syncthreads();
  const int G = max(1, min(32, nt / k));
  for (int round = 0; round < 40; ++round) {
    const int i = tid / G, g = tid % G;
    if (i < k) {
      const float a = flo[i], b = fhi[i];
      const float x = a + (b - a) * (float)(g + 1) / (float)(G + 1);
      icnt[tid] = (b - a > 4e-7f * fmaxf(fabsf(a), fabsf(b)) + 1e-30f) ? sturm_count_f32(n, df, e2f, x) : -1;
    }
    __syncthreads();
    int moved = 0;
    if (i < k && g == 0 && icnt[tid] >= 0) {
      const float a = flo[i], b = fhi[i];
      float na = a, nb = b;
      for (int q = 0; q < G; ++q) {
        const float x = a + (b - a) * (float)(q + 1) / (float)(G + 1);
        if (icnt[i * G + q] > i) {
          nb = x;
          break;
        }
        na = x;
      }
      flo[i] = na;
      fhi[i] = nb;
      moved = 1;
    }
    if (block_sum((double)moved, red) == 0.0) break;
  }
  for (int i = tid; i < k; i += nt) W.lamx[i] = 0.5 * ((double)flo[i] + (double)fhi[i]);
  if (tid == 0) W.lamx[k] = fmax(fabs(s_lo), fabs(s_hi));
}

// 4. inverse iteration, one CTA per eigenvalue (only cluster heads work; lane 0 runs the
//    sequential recurrences on shared-memory scratch).  Eigenvalues closer than
//    ctol = 1e-5 |T| form a cluster: its vectors are re-orthogonalised against each other
//    (vectors of close eigenvalues computed independently lose orthogonality by
//    ~eps |T| / gap) and rotated by a Rayleigh-Ritz step inside the cluster.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Largest number of vectors of one cluster iterated side by side (one lane each); each
// lane keeps its tridiagonal-solve scratch (4n doubles, padded by one) in shared memory.
__host__ __device__ inline int inviter_lanes(int n) {
  const int budget = 160 * 1024;
  int l = budget / ((4 * n + 1) * (int)sizeof(double));
  return l < 1 ? 1 : (l > 32 ? 32 : l);
}

// One warp per cluster head: inverse iteration with Rayleigh-quotient shifts for the
// eigenvalues of the cluster, run for up to inviter_lanes(n) vectors at once (lane j
// solves with vector j's own shift), each sweep followed by modified Gram-Schmidt of the
// block against the cluster's earlier vectors and within itself; then a Jacobi
// Rayleigh-Ritz inside the cluster.  Dot products, updates, norms and Rayleigh quotients
// are spread over the 32 lanes.
__global__ void __launch_bounds__(32) k_sygv_inviter(int n, int k, double* work, double* __restrict__ lam,
                                                     const int* status) {
  if (status[0] != 0) return;
  extern __shared__ double sw[];  // inviter_lanes(n) x (4n + 1)
  __shared__ double H[kClusterRR * kClusterRR], R[kClusterRR * kClusterRR];
  __shared__ double shifts[32];
  __shared__ int perm[kClusterRR];
  SygvWork W = sygv_work(work, n, k);
  const int i = blockIdx.x, lane = threadIdx.x;
  const double tnorm = W.lamx[k];
  const double ctol = 1e-5 * tnorm;
  const double tiny = DBL_EPSILON * tnorm + DBL_MIN;
  const double* lx = W.lamx;
  if (i > 0 && lx[i] - lx[i - 1] <= ctol) return;  // not a cluster head (uniform per block)
  int last = i;
  while (last + 1 < k && lx[last + 1] - lx[last] <= ctol) ++last;
  const double* d = W.d;
  const double* e = W.e;
  double* Z = W.Z;
  const int SP = inviter_lanes(n);
  const int ld = 4 * n + 1;
  auto vec = [&](int j) { return sw + (size_t)j * ld + 3 * n; };  // vector j of the block
  for (int c0 = i; c0 <= last; c0 += SP) {
    const int cs = min(SP, last + 1 - c0);
    for (int j = 0; j < cs; ++j)
      for (int r = lane; r < n; r += 32) vec(j)[r] = hash_unit((unsigned)(c0 + j), (unsigned)r) + 1e-3;
    if (lane < cs) shifts[lane] = lx[c0 + lane];
    const int iters = (i == last) ? 3 : 4;
    for (int it = 0; it < iters; ++it) {
      __syncwarp();
      if (lane < cs) {
        double* base = sw + (size_t)lane * ld;
        tri_solve(n, d, e, shifts[lane], base + 3 * n, base, base + n, base + 2 * n, tiny);
      }
      __syncwarp();
      for (int j = 0; j < cs; ++j) {
        double* b = vec(j);
        for (int pass = 0; pass < 2; ++pass) {
          for (int o = i; o < c0; ++o) {  // earlier chunks of the cluster (in Z)
            double dot = 0.0;
            for (int r = lane; r < n; r += 32) dot = fma(b[r], Z[(int64_t)r * k + o], dot);
            dot = warp_sum(dot);
            for (int r = lane; r < n; r += 32) b[r] -= dot * Z[(int64_t)r * k + o];
          }
          for (int o = 0; o < j; ++o) {  // earlier vectors of this block
            const double* bo = vec(o);
            double dot = 0.0;
            for (int r = lane; r < n; r += 32) dot = fma(b[r], bo[r], dot);
            dot = warp_sum(dot);
            for (int r = lane; r < n; r += 32) b[r] -= dot * bo[r];
          }
        }
        double nrm = 0.0;
        for (int r = lane; r < n; r += 32) nrm = fma(b[r], b[r], nrm);
        nrm = warp_sum(nrm);
        const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
        for (int r = lane; r < n; r += 32) b[r] *= inv;
        __syncwarp();
        if (it >= 1) {  // Rayleigh-quotient shift
          double rq = 0.0;
          for (int r = lane; r < n; r += 32) {
            double tq = d[r] * b[r];
            if (r > 0) tq += e[r - 1] * b[r - 1];
            if (r < n - 1) tq += e[r] * b[r + 1];
            rq = fma(b[r], tq, rq);
          }
          rq = warp_sum(rq);
          if (lane == 0) shifts[j] = rq;
        }
        __syncwarp();
      }
    }
    if (lane < cs) lam[c0 + lane] = shifts[lane];
    for (int j = 0; j < cs; ++j)
      for (int r = lane; r < n; r += 32) Z[(int64_t)r * k + c0 + j] = vec(j)[r];
    __syncwarp();
  }
  const int s = last - i + 1;
  if (s >= 2 && s <= kClusterRR) {
    // projected tridiagonal matrix of the cluster's vectors
    for (int a = 0; a < s; ++a)
      for (int b = a; b < s; ++b) {
        double acc = 0.0;
        for (int r = lane; r < n; r += 32) {
          double tq = d[r] * Z[(int64_t)r * k + i + b];
          if (r > 0) tq += e[r - 1] * Z[(int64_t)(r - 1) * k + i + b];
          if (r < n - 1) tq += e[r] * Z[(int64_t)(r + 1) * k + i + b];
          acc = fma(Z[(int64_t)r * k + i + a], tq, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
          H[a * s + b] = acc;
          H[b * s + a] = acc;
        }
      }
    __syncwarp();
    if (lane == 0) {  // cyclic Jacobi on the s x s matrix (s <= 16)
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) R[a * s + b] = (a == b) ? 1.0 : 0.0;
      for (int sweep = 0; sweep < 12; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int a = 0; a < s; ++a) {
          diag += H[a * s + a] * H[a * s + a];
          for (int b = a + 1; b < s; ++b) off += H[a * s + b] * H[a * s + b];
        }
        if (off <= 1e-30 * (diag + DBL_MIN)) break;
        for (int a = 0; a < s; ++a)
          for (int b = a + 1; b < s; ++b) {
            const double hab = H[a * s + b];
            if (hab == 0.0) continue;
            const double th = 0.5 * (H[b * s + b] - H[a * s + a]) / hab;
            const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double c = 1.0 / sqrt(tt * tt + 1.0), sn = tt * c;
            for (int l = 0; l < s; ++l) {
              const double ha = H[l * s + a], hb = H[l * s + b];
              H[l * s + a] = c * ha - sn * hb;
              H[l * s + b] = sn * ha + c * hb;
            }
            for (int l = 0; l < s; ++l) {
              const double ha = H[a * s + l], hb = H[b * s + l];
              H[a * s + l] = c * ha - sn * hb;
              H[b * s + l] = sn * ha + c * hb;
            }
            for (int l = 0; l < s; ++l) {
              const double ra = R[l * s + a], rb = R[l * s + b];
              R[l * s + a] = c * ra - sn * rb;
              R[l * s + b] = sn * ra + c * rb;
            }
          }
      }
      for (int a = 0; a < s; ++a) perm[a] = a;
      for (int a = 0; a < s; ++a)
        for (int b = a + 1; b < s; ++b)
          if (H[perm[b] * s + perm[b]] < H[perm[a] * s + perm[a]]) {
            const int t2 = perm[a];
            perm[a] = perm[b];
            perm[b] = t2;
          }
    }
    __syncwarp();
    for (int r = lane; r < n; r += 32) {  // rotate the cluster's rows (one row per lane)
      double row[kClusterRR];
      for (int a = 0; a < s; ++a) {
        double acc = 0.0;
        for (int b = 0; b < s; ++b) acc += Z[(int64_t)r * k + i + b] * R[b * s + perm[a]];
        row[a] = acc;
      }
      for (int a = 0; a < s; ++a) Z[(int64_t)r * k + i + a] = row[a];
    }
    if (lane < s) lam[i + lane] = H[perm[lane] * s + perm[lane]];
  }
}

// 3b. Householder tridiagonalisation on a thread-block cluster of kTriC CTAs (one SM
//     each): CTA c keeps the full rows r = c, c + kTriC, ... of the symmetric matrix in
//     its shared memory.  Step j: each CTA computes p = t A22 v for its own rows and
//     writes those entries (and its share of p.v) into every CTA (one cluster barrier);
//     every CTA then applies the rank-2 update to its own rows, the owner of row j+1 that
//     row first, from which it forms reflector j+1 (as kernel 3) and writes it into every
//     CTA before arriving on a split cluster barrier; the other rows' updates run before
//     the wait.  Reflector, p and partial sums are double buffered by step parity.  d, e,
//     tau and the reflectors go to the workspace exactly as in kernel 3; the eigenvalue
//     brackets are computed afterwards by k_sygv_multisect.
//     The cluster has kTriC CTAs (portable size) or 2 kTriC (a non-portable size, where
//     the part can schedule it); the launch sets the cluster shape.
constexpr int kTriC = 8;
constexpr int kTriClusterMin = 64;  // default: below this the single-CTA kernels (the autotuner may choose)
__host__ __device__ inline size_t tri_cluster_smem(int n, int C) {
  const int rows = (n + C - 1) / C;
  return ((size_t)rows * n + 4 * (size_t)n + 4 * C + 8) * sizeof(double);
}

template <int C>
__global__ void __launch_bounds__(256) k_sygv_tridiag_c(int n, int k, double* work, const int* status) {
  constexpr int kTriC = C;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  if (status[0] != 0) return;  // uniform over the cluster (written by an earlier kernel)
  extern __shared__ double smc[];
  __shared__ double red[40];
  SygvWork W = sygv_work(work, n, k);
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  const int nrows = (n - rank + kTriC - 1) / kTriC;  // rows owned by this CTA
  double* Arow = smc;                                           // [nrows][n]
  double* vb = Arow + (size_t)((n + kTriC - 1) / kTriC) * n;    // [2][n] reflector
  double* pb = vb + 2 * n;                                      // [2][n] p
  double* part = pb + 2 * n;                                    // [2][kTriC] partial p.v
  double* scal = part + 2 * kTriC;                              // [2][2] t, beta; [4..] max exchange
  const double* K = W.K;
  for (int lr = warp; lr < nrows; lr += nwarps) {
    const int r = lr * kTriC + rank;
    for (int c = lane; c < n; c += 32) Arow[(size_t)lr * n + c] = 0.5 * (K[(int64_t)r * n + c] + K[(int64_t)c * n + r]);
  }
  __syncthreads();
  if (W.info[0] > 0) {  // dropped directions get a value above the kept spectrum
    double rmax = 0.0;
    for (int lr = tid; lr < nrows; lr += nt) {
      const int r = lr * kTriC + rank;
      if (W.tau[r] != 0.0) continue;
      double a = 0.0;
      for (int c = 0; c < n; ++c)
        if (W.tau[c] == 0.0) a += fabs(Arow[(size_t)lr * n + c]);
      rmax = fmax(rmax, a);
    }
    rmax = block_max(rmax, red);
    if (tid < kTriC) *cluster.map_shared_rank(scal + 4 + rank, tid) = rmax;
    cluster.sync();
    double big = 0.0;
    for (int q = 0; q < kTriC; ++q) big = fmax(big, scal[4 + q]);
    big = 2.0 * big + 1.0;
    for (int lr = warp; lr < nrows; lr += nwarps) {
      const int r = lr * kTriC + rank;
      for (int c = lane; c < n; c += 32)
        if (W.tau[r] != 0.0 || W.tau[c] != 0.0) Arow[(size_t)lr * n + c] = (r == c) ? big : 0.0;
    }
  }
  cluster.sync();  // the drop mask in tau is read above and overwritten below
  // reflector j from row j (kernel 3's form), written into every CTA with its t and beta;
  // a step of the whole owner CTA
  __shared__ double s_hh[3];
  auto reflector = [&](int j) {
    const int par = j & 1;
    const int len = n - j - 1, j1 = j + 1;
    double* v = vb + par * n;
    double* sc = scal + par * 2;
    const double* x = Arow + (size_t)(j / kTriC) * n + j1;
    double ps = 0.0;
    for (int r = 1 + tid; r < len; r += nt) ps += x[r] * x[r];
    const double sig = block_sum(ps, red);
    if (tid == 0) {
      const double x0 = x[0];
      double beta = x0, t = 0.0, sl = 0.0;
      if (sig != 0.0) {
        const double nrm = sqrt(x0 * x0 + sig);
        beta = (x0 >= 0.0) ? -nrm : nrm;
        t = (beta - x0) / beta;
        sl = 1.0 / (x0 - beta);
      }
      s_hh[0] = beta;
      s_hh[1] = t;
      s_hh[2] = sl;
      W.d[j] = Arow[(size_t)(j / kTriC) * n + j];
      W.e[j] = beta;
      W.tau[j] = t;
    }
    __syncthreads();
    const double t = s_hh[1], sl = s_hh[2];
    for (int r = tid; r < len; r += nt) {
      const double vr = (r == 0) ? 1.0 : x[r] * sl;
      if (r >= 1) W.K[(int64_t)j * n + (j1 + r)] = vr;  // reflector store
      for (int q = 0; q < kTriC; ++q) *cluster.map_shared_rank(v + r, q) = vr;
    }
    if (tid < kTriC) {
      *cluster.map_shared_rank(sc, tid) = t;
      *cluster.map_shared_rank(sc + 1, tid) = s_hh[0];
    }
  };
  if (rank == 0 && n > 2) reflector(0);
  cluster.sync();
  // Step j: p = t A22 v and p.v over the cluster (one barrier); then the owner of row j+1
  // applies the rank-2 update to that row alone, forms reflector j+1 and arrives on the
  // split cluster barrier while every CTA applies the update to its other rows, so the
  // reflector's exchange overlaps the update.  v, p and the partial sums are double
  // buffered by step parity.
  for (int j = 0; j + 2 < n; ++j) {
    const int par = j & 1;
    const int len = n - j - 1, j1 = j + 1;
    double* v = vb + par * n;
    double* pp = pb + par * n;
    double* pt = part + par * kTriC;
    double* sc = scal + par * 2;
    const double t = sc[0];
    if (t != 0.0) {
      // p = t A22 v for this CTA's rows R >= j1; share of p.v
      double pvp = 0.0;
      const int lr0 = (j1 - rank + kTriC - 1) / kTriC;  // first own local row with R >= j1
      for (int lr = lr0 + warp; lr < nrows; lr += nwarps) {
        const int R = lr * kTriC + rank;
        const double* row = Arow + (size_t)lr * n + j1;
        double acc = 0.0;
        for (int c = lane; c < len; c += 32) acc = fma(row[c], v[c], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double pr = t * acc;
        if (lane < kTriC) *cluster.map_shared_rank(pp + (R - j1), lane) = pr;
        if (lane == 0) pvp += pr * v[R - j1];
      }
      const double pvs = block_sum(pvp, red);
      if (tid < kTriC) *cluster.map_shared_rank(pt + rank, tid) = pvs;
    }
    cluster.sync();
    const bool next = j + 3 < n;                              // a reflector j+1 follows
    const bool owner_next = next && (j1 % kTriC == rank);     // this CTA forms it
    if (t != 0.0) {
      double pv = 0.0;
      for (int q = 0; q < kTriC; ++q) pv += pt[q];
      const double Kc = 0.5 * t * pv;
      for (int r = tid; r < len; r += nt) pp[r] -= Kc * v[r];
      __syncthreads();
      if (owner_next) {  // row j+1 first
        double* row = Arow + (size_t)(j1 / kTriC) * n + j1;
        const double vR = v[0], pR = pp[0];
        for (int c = tid; c < len; c += nt) row[c] -= vR * pp[c] + pR * v[c];
        __syncthreads();
      }
    }
    if (owner_next) reflector(j1);
    if (next) asm volatile("barrier.cluster.arrive.release;" ::: "memory");
    if (t != 0.0) {
      const int lr0 = (j1 - rank + kTriC - 1) / kTriC;
      for (int lr = lr0 + warp; lr < nrows; lr += nwarps) {
        const int R = lr * kTriC + rank;
        if (owner_next && R == j1) continue;  // done above
        double* row = Arow + (size_t)lr * n + j1;
        const double vR = v[R - j1], pR = pp[R - j1];
        for (int c = lane; c < len; c += 32) row[c] -= vR * pp[c] + pR * v[c];
      }
    }
    __syncthreads();  // own rows complete before the next step's products read them
    if (next) asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
  }
  // the trailing 2 x 2 block
  if (tid == 0) {
    if (n >= 2 && (n - 2) % kTriC == rank) {
      W.d[n - 2] = Arow[(size_t)((n - 2) / kTriC) * n + (n - 2)];
      W.tau[n - 2] = 0.0;
    }
    if ((n - 1) % kTriC == rank) {
      if (n >= 2) W.e[n - 2] = Arow[(size_t)((n - 1) / kTriC) * n + (n - 2)];
      W.d[n - 1] = Arow[(size_t)((n - 1) / kTriC) * n + (n - 1)];
      W.e[n - 1] = 0.0;
      W.tau[n - 1] = 0.0;
    }
  }
  cluster.sync();  // no CTA leaves while another may still address its shared memory
}

// 1c. Scaling + Cholesky with dropping (the result of kernel 1) on a thread-block cluster
//     of C CTAs (one SM each, launch-set cluster shape): CTA c keeps the lower parts of rows
//     r = c, c + C, ... in shared memory.  Step j (right-looking, unscaled: a_rc -= a_rj
//     a_cj / d_j over j < c <= r, d_j the pivot): every CTA first updates column j+1 of its
//     own rows and writes those entries (and, on the owner of row j+1, the next pivot's
//     reciprocal) into every CTA, arrives on the cluster barrier, applies the rest of the
//     step to its own rows, and waits; so the barrier's latency hides behind the update.
//     Columns rotate through three buffers, which keeps a fast CTA's writes off a buffer
//     a slow one still reads.  L = a_rj / sqrt(d_j) is formed once at the end.  The drop
//     rule, outputs and status are those of kernel 1.
__host__ __device__ inline size_t chol_cluster_smem(int n, int C) {
  const int rows = (n + C - 1) / C;
  return ((size_t)rows * n + 7 * (size_t)n + 4) * sizeof(double);
}

template <int C>
__global__ void __launch_bounds__(256) k_sygv_chol_c(int n, int k, const double* __restrict__ GA, int lda,
                                                     const double* __restrict__ GB, int ldb, double* work,
                                                     int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double smh[];
  __shared__ int s_fail;
  SygvWork W = sygv_work(work, n, k);
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  const int nrows = (n - rank + C - 1) / C;  // rows owned by this CTA
  double* Ar = smh;                                      // [rows][n], lower parts
  double* cb = Ar + (size_t)((n + C - 1) / C) * n;       // [3][n] column j (unscaled)
  double* sc = cb + 3 * (size_t)n;                       // [n] diagonal scaling
  double* piv = sc + n;                                  // [n] pivots d_j
  double* sq = piv + n;                                  // [n] sqrt(d_j) (1 if dropped)
  double* rs = sq + n;                                   // [n] 1 / sqrt(d_j) (0 if dropped)
  double* rdb = rs + n;                                  // [3] 1 / d_j (0 if dropped)
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int i = tid; i < n; i += nt) {  // every CTA checks every pivot, so all leave together
    const double g = GB[(int64_t)i * ldb + i];
    if (!(g >= 0.0) || !isfinite(g)) s_fail = 1;
    sc[i] = (g > 0.0) ? rsqrt(g) : 0.0;
  }
  __syncthreads();
  if (s_fail) {
    if (rank == 0 && tid == 0) status[0] = 1;
    return;
  }
  if (rank == 0)
    for (int i = tid; i < n; i += nt) W.sc[i] = sc[i];
  for (int lr = warp; lr < nrows; lr += nwarps) {
    const int r = lr * C + rank;
    for (int c = lane; c < n; c += 32) {
      const double t = sc[r] * sc[c];
      W.K[(int64_t)r * n + c] = t * 0.5 * (GA[(int64_t)r * lda + c] + GA[(int64_t)c * lda + r]);
      if (c <= r) Ar[(size_t)lr * n + c] = t * 0.5 * (GB[(int64_t)r * ldb + c] + GB[(int64_t)c * ldb + r]);
    }
  }
  __syncthreads();
  for (int lr = tid; lr < nrows; lr += nt) {  // column 0 and the first pivot to every CTA
    const int r = lr * C + rank;
    const double v = Ar[(size_t)lr * n];
    for (int q = 0; q < C; ++q) *cluster.map_shared_rank(cb + r, q) = v;
    if (r == 0) {
      const double rd = (v > kPivTol && isfinite(v)) ? fast_rcp(v) : 0.0;
      for (int q = 0; q < C; ++q) *cluster.map_shared_rank(rdb, q) = rd;
    }
  }
  cluster.sync();
  for (int j = 0; j < n; ++j) {
    const double* col = cb + (size_t)(j % 3) * n;
    const double rdj = rdb[j % 3];
    const bool drop = rdj == 0.0;
    if (tid == 0) piv[j] = col[j];
    if (j + 1 < n) {
      // column j+1 of the own rows r >= j+1, then to every CTA
      double* nxt = cb + (size_t)((j + 1) % 3) * n;
      const double t = col[j + 1] * rdj;
      const int lr0 = (j + 1 - rank + C - 1) / C;
      for (int lr = lr0 + tid; lr < nrows; lr += nt) {
        const int r = lr * C + rank;
        double v = Ar[(size_t)lr * n + j + 1];
        if (!drop) v = fma(-col[r], t, v);
        Ar[(size_t)lr * n + j + 1] = v;
        for (int q = 0; q < C; ++q) *cluster.map_shared_rank(nxt + r, q) = v;
        if (r == j + 1) {
          const double rd = (v > kPivTol && isfinite(v)) ? fast_rcp(v) : 0.0;
          for (int q = 0; q < C; ++q) *cluster.map_shared_rank(rdb + (j + 1) % 3, q) = rd;
        }
      }
      asm volatile("barrier.cluster.arrive.release;" ::: "memory");
    }
    // the rest of step j on the own rows r >= j+2: columns j+2 .. r
    if (!drop) {
      const int lr0 = (j + 2 - rank + C - 1) / C;
      for (int lr = lr0 + warp; lr < nrows; lr += nwarps) {
        const int r = lr * C + rank;
        double* row = Ar + (size_t)lr * n;
        const double tr = col[r] * rdj;
        for (int c = j + 2 + lane; c <= r; c += 32) row[c] = fma(-tr, col[c], row[c]);
      }
    }
    __syncthreads();  // own rows complete before the next step's column update reads them
    if (j + 1 < n) asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
  }
  // L from the unscaled columns: L_rc = a_rc / sqrt(d_c), L_cc = sqrt(d_c); dropped: 0, 1
  int nd = 0;
  for (int c = tid; c < n; c += nt) {
    const double d = piv[c];
    const bool dr = !(d > kPivTol) || !isfinite(d);
    sq[c] = dr ? 1.0 : sqrt(d);
    rs[c] = dr ? 0.0 : 1.0 / sq[c];
    if (rank == 0) W.tau[c] = dr ? 1.0 : 0.0;
    nd += dr ? 1 : 0;
  }
  __syncthreads();
  for (int lr = warp; lr < nrows; lr += nwarps) {
    const int r = lr * C + rank;
    for (int c = lane; c < n; c += 32) {
      const double v = (c < r) ? Ar[(size_t)lr * n + c] * rs[c] : (c == r ? sq[r] : 0.0);
      W.L[(int64_t)r * n + c] = v;
    }
  }
  if (rank == 0) {
    __shared__ double red[40];
    const double ndrop = block_sum((double)nd, red);
    if (tid == 0) {
      W.info[0] = (int)ndrop;
      status[0] = (n - (int)ndrop < k) ? 1 : 0;
    }
  }
  cluster.sync();  // no CTA leaves while another may still address its shared memory
}

// 3c. Gershgorin bounds of the tridiagonal matrix and FP32 multisection for the k
//     smallest eigenvalues (the tail of kernel 3, for the cluster variant).
__global__ void __launch_bounds__(1024) k_sygv_multisect(int n, int k, double* work, const int* status) {
  if (status[0] != 0) return;
  extern __shared__ double shm[];
  __shared__ double red[40];
  __shared__ double s_lo, s_hi;
  SygvWork W = sygv_work(work, n, k);
  const int tid = threadIdx.x, nt = blockDim.x;
  int* icnt = reinterpret_cast<int*>(shm);  // nt
  float* df = reinterpret_cast<float*>(icnt + nt);
  float* e2f = df + n;
  float* flo = e2f + n;
  float* fhi = flo + k;
  if (tid == 0) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(W.e[i - 1]) : 0.0) + (i < n - 1 ? fabs(W.e[i]) : 0.0);
      lo = fmin(lo, W.d[i] - r);
      hi = fmax(hi, W.d[i] + r);
    }
    s_lo = lo;
    s_hi = hi;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    df[i] = (float)W.d[i];
    e2f[i] = (float)(W.e[i] * W.e[i]);
  }
  for (int i = tid; i < k; i += nt) {
    flo[i] = (float)s_lo - 1e-6f * (float)fabs(s_lo) - 1e-30f;
    fhi[i] = (float)s_hi + 1e-6f * (float)fabs(s_hi) + 1e-30f;
  }
  __syncthreads();
  const int G = max(1, min(32, nt / k));
  for (int round = 0; round < 40; ++round) {
    const int i = tid / G, g = tid % G;
    if (i < k) {
      const float a = flo[i], b = fhi[i];
      const float x = a + (b - a) * (float)(g + 1) / (float)(G + 1);
      icnt[tid] = (b - a > 4e-7f * fmaxf(fabsf(a), fabsf(b)) + 1e-30f) ? sturm_count_f32(n, df, e2f, x) : -1;
    }
    __syncthreads();
    int moved = 0;
    if (i < k && g == 0 && icnt[tid] >= 0) {
      const float a = flo[i], b = fhi[i];
      float na = a, nb = b;
      for (int q = 0; q < G; ++q) {
        const float x = a + (b - a) * (float)(q + 1) / (float)(G + 1);
        if (icnt[i * G + q] > i) {
          nb = x;
          break;
        }
        na = x;
      }
      flo[i] = na;
      fhi[i] = nb;
      moved = 1;
    }
    if (block_sum((double)moved, red) == 0.0) break;
  }
  for (int i = tid; i < k; i += nt) W.lamx[i] = 0.5 * ((double)flo[i] + (double)fhi[i]);
  if (tid == 0) W.lamx[k] = fmax(fabs(s_lo), fabs(s_hi));  // |T| bound
}

// 5. back-transform: one CTA per column of Z; its four warps stage the reflectors (then
//    L) in shared memory and warp 0 takes the column through z <- H_0 ... H_{n-3} z, then
//    c = D L^-T z.  One column per CTA spreads the FP64 work of the k columns over k SMs.
constexpr int kBtThreads = 128;
__global__ void __launch_bounds__(kBtThreads) k_sygv_back(int n, int k, double* work, double* __restrict__ C,
                                                         int ldc, int stage, const int* status) {
  // the reflector sweep and the triangular solve are sequences of n dependent steps, each
  // a dot product and an update over one column: one warp runs them with shuffles
  if (status[0] != 0) return;
  extern __shared__ double zc[];  // z [n], reciprocal pivots [n], then [packed reflectors | packed L]
  SygvWork W = sygv_work(work, n, k);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  double* z = zc;
  double* rinv = zc + n;
  double* pk = zc + 2 * n;
  const int col = blockIdx.x;
  for (int r = tid; r < n; r += blockDim.x) {
    z[r] = W.Z[(int64_t)r * k + col];
    rinv[r] = 1.0 / W.L[(int64_t)r * n + r];
  }
  // reflector j (rows j+1..n-1): v[0] = 1, v[r] = K[j][j+1+r] for r >= 1, packed at
  // pk + off(j), off(j) = j(n-2) - j(j-1)/2, n-j-2 entries
  if (stage) {
    for (int j = warp; j + 2 < n; j += nwarps) {
      const int off = j * (n - 2) - j * (j - 1) / 2;
      for (int r = lane; r < n - j - 2; r += 32) pk[off + r] = W.K[(int64_t)j * n + (j + 2 + r)];
    }
  }
  __syncthreads();
  if (warp == 0) {
    for (int j = n - 3; j >= 0; --j) {
      const double t = W.tau[j];
      if (t == 0.0) continue;
      const int len = n - j - 1;
      const double* vr = stage ? pk + (j * (n - 2) - j * (j - 1) / 2) - 1 : W.K + (int64_t)j * n + (j + 1);
      double acc = 0.0;
      for (int r = lane; r < len; r += 32) acc = fma(r == 0 ? 1.0 : vr[r], z[j + 1 + r], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const double c = t * acc;
      for (int r = lane; r < len; r += 32) z[j + 1 + r] -= c * (r == 0 ? 1.0 : vr[r]);
      __syncwarp();
    }
  }
  // L^T x = z, rows from the bottom (column i of L = L[l][i], l > i); L packed by rows,
  // row l at off(l) = l(l+1)/2, when staged
  if (stage) {
    __syncthreads();  // the reflector sweep is done
    for (int l = warp; l < n; l += nwarps)
      for (int c = lane; c <= l; c += 32) pk[l * (l + 1) / 2 + c] = W.L[(int64_t)l * n + c];
    __syncthreads();
  }
  if (warp != 0) return;
  __syncwarp();
  // column-oriented back substitution: lane l % 32 owns z[l]; step i takes x_i = z_i / L_ii
  // on its owner lane, broadcasts it, and every lane takes L[i][l] x_i off its rows l < i
  for (int i = n - 1; i >= 0; --i) {
    const double xi = __shfl_sync(0xffffffffu, z[i] * rinv[i], i & 31);
    if (lane == (i & 31)) z[i] = xi;
    for (int l = lane; l < i; l += 32) {
      const double lil = stage ? pk[i * (i + 1) / 2 + l] : W.L[(int64_t)i * n + l];
      z[l] = fma(-lil, xi, z[l]);
    }
  }
  __syncwarp();
  for (int r = lane; r < n; r += 32) C[(int64_t)r * ldc + col] = W.sc[r] * z[r];
}

size_t small_sygv_work_doubles(int n, int k) {
  return (size_t)3 * n * n + (size_t)n * k + 4 * (size_t)n + k + 8;
}

// Launch one of the cluster kernels (k_sygv_chol_c, k_sygv_tridiag_c) as a single cluster
// of csize CTAs of 256 threads.
template <typename... KArgs, typename... Args>
static int launch_sygv_cluster(void (*kern)(KArgs...), int csize, size_t smem, cudaStream_t s, Args... args) {
  PASE_TRY(ensure_max_smem((const void*)kern, 200 * 1024));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)csize, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  PASE_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
  return PASE_OK;
}

// Whether this device schedules one cluster of 2 kTriC CTAs of the tridiagonalisation
// (a non-portable cluster size), asked once per device.
static bool tri16_available(int device, size_t smem) {
  static std::mutex mu;
  static int avail[64];
  static bool init = false;
  std::lock_guard<std::mutex> lk(mu);
  if (!init) {
    for (int& a : avail) a = -1;
    init = true;
  }
  if (device < 0 || device >= 64) return false;
  if (avail[device] < 0) {
    int ok = 0;
    const void* f = (const void*)k_sygv_tridiag_c<2 * kTriC>;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        ensure_max_smem(f, 200 * 1024) == PASE_OK) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2 * kTriC, 1, 1);
      cfg.blockDim = dim3(256, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2 * kTriC;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, k_sygv_tridiag_c<2 * kTriC>, &cfg) == cudaSuccess && nc >= 1) ok = 1;
    }
    cudaGetLastError();
    avail[device] = ok;
  }
  return avail[device] == 1;
}

int small_sygv(pase_ctx* h, int n, int k, const double* GA, int lda, const double* GB, int ldb,
               double* lam, double* C, int ldc, int* status_dev) {
  if (n <= 0 || k <= 0 || k > n || k > 1024) return fail(PASE_ERR_INVALID_ARG, "small_sygv: bad size");
  // threads of the single-CTA stages (Cholesky, tridiagonalisation, multisection): the
  // FP64 pipe of one SM bounds them, so fewer threads (cheaper barriers) can be faster;
  // the autotuner picks per size, at least k (one multisection lane per eigenvalue)
  int thr = 1024;
  // tridiagonalisation: 0 one CTA, 1 a cluster of kTriC SMs, 2 of 2 kTriC SMs; Cholesky:
  // 0 one CTA, 1 a cluster of kTriC SMs
  int tform = n >= kTriClusterMin ? 1 : 0;
  int cform = n >= kTriClusterMin ? 1 : 0;
  for (int i = 0; i < 3; ++i)
    if (h->sygv_n[i] == n) {
      if (h->sygv_thr[i] >= k) thr = h->sygv_thr[i];
      if (h->sygv_cl[i] >= 0 && n >= 16) tform = h->sygv_cl[i];
      if (h->sygv_ch[i] >= 0 && n >= 16) cform = h->sygv_ch[i];
    }
  if (h->opt.sygv_tridiag >= 0) tform = n >= 16 ? h->opt.sygv_tridiag : 0;  // fixed by the caller
  if (h->opt.sygv_cholesky >= 0) cform = n >= 16 ? h->opt.sygv_cholesky : 0;
  if (small_sygv_work_doubles(n, k) > h->w.eigwork_doubles)
    return fail(PASE_ERR_INVALID_ARG, "small_sygv: workspace too small");
  const size_t smem_tri = (size_t)(2 * n + 1024) * sizeof(double) + 1024 * sizeof(int) + (size_t)(2 * n + 2 * k) * sizeof(float);
  if (smem_tri > 200 * 1024 || (size_t)4 * n * sizeof(double) > 200 * 1024)
    return fail(PASE_ERR_INVALID_ARG, "small_sygv: problem too large");
  for (const void* f : {(const void*)k_sygv_tridiag, (const void*)k_sygv_inviter, (const void*)k_sygv_back,
                        (const void*)k_sygv_trsm, (const void*)k_sygv_chol_s, (const void*)k_sygv_tridiag_s})
    PASE_TRY(ensure_max_smem(f, 200 * 1024));
  double* w = h->w.eigwork;
  auto s = h->stream;
  const size_t tri = (size_t)n * (n + 1) / 2;
  // columns per CTA of the triangular solves: one wave of the SMs (at most 4, one warp each)
  const int cpc = std::min(4, std::max(1, (n + h->num_sms - 1) / h->num_sms));
  const int trsm_grid = (n + cpc - 1) / cpc;
  const size_t smem_trsm_st = (size_t)((2 * cpc + 1) * n + tri) * sizeof(double);
  const int stage_l = smem_trsm_st <= 200 * 1024 ? 1 : 0;
  const size_t smem_trsm = stage_l ? smem_trsm_st : (size_t)((2 * cpc + 1) * n) * sizeof(double);
  const size_t smem_back_st = (size_t)(2 * n + tri) * sizeof(double);
  const int stage_b = smem_back_st <= 200 * 1024 ? 1 : 0;
  const size_t smem_back = stage_b ? smem_back_st : (size_t)2 * n * sizeof(double);
  const size_t smem_chol_s = (tri + n) * sizeof(double);
  const size_t smem_tri_s = (tri + 2 * n) * sizeof(double) + 1024 * sizeof(int) + (size_t)(2 * n + 2 * k) * sizeof(float);
  const bool packed = smem_tri_s <= 200 * 1024 && smem_chol_s <= 200 * 1024;
  const size_t smem_chc = chol_cluster_smem(n, kTriC);
  if (cform == 1 && smem_chc <= 200 * 1024)
    PASE_TRY(launch_sygv_cluster(k_sygv_chol_c<kTriC>, kTriC, smem_chc, s, n, k, GA, lda, GB, ldb, w, status_dev));
  else if (packed)
    k_sygv_chol_s<<<1, thr, smem_chol_s, s>>>(n, k, GA, lda, GB, ldb, w, status_dev);
  else
    k_sygv_chol<<<1, thr, (size_t)n * sizeof(double), s>>>(n, k, GA, lda, GB, ldb, w, status_dev);
  k_sygv_trsm<<<trsm_grid, 128, smem_trsm, s>>>(n, k, w, 0, stage_l, cpc, status_dev);
  k_sygv_trsm<<<trsm_grid, 128, smem_trsm, s>>>(n, k, w, 1, stage_l, cpc, status_dev);
  const size_t smem_c = tri_cluster_smem(n, kTriC), smem_c2 = tri_cluster_smem(n, 2 * kTriC);
  const size_t smem_ms = (size_t)1024 * sizeof(int) + (size_t)(2 * n + 2 * k) * sizeof(float);
  if (tform == 2 && (smem_c2 > 200 * 1024 || !tri16_available(h->device, smem_c2))) tform = 1;
  if (tform >= 1 && smem_c <= 200 * 1024) {  // reduction spread over a cluster of SMs
    if (tform == 2)
      PASE_TRY(launch_sygv_cluster(k_sygv_tridiag_c<2 * kTriC>, 2 * kTriC, smem_c2, s, n, k, w,
                                   (const int*)status_dev));
    else
      PASE_TRY(launch_sygv_cluster(k_sygv_tridiag_c<kTriC>, kTriC, smem_c, s, n, k, w, (const int*)status_dev));
    k_sygv_multisect<<<1, thr, smem_ms, s>>>(n, k, w, status_dev);
    h->launches++;
  } else if (packed) {
    k_sygv_tridiag_s<<<1, thr, smem_tri_s, s>>>(n, k, w, status_dev);
  } else {
    k_sygv_tridiag<<<1, thr, smem_tri, s>>>(n, k, w, status_dev);
  }
  k_sygv_inviter<<<k, 32, (size_t)inviter_lanes(n) * (4 * n + 1) * sizeof(double), s>>>(n, k, w, lam, status_dev);
  k_sygv_back<<<k, kBtThreads, smem_back, s>>>(n, k, w, C, ldc, stage_b, status_dev);
  h->launches += 6;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

}  // namespace pase

namespace pase {

// ------------------------------------------------------------------ dense helpers (batch scheme)
// Row r of a CSR matrix into row r of a dense row-major block (zeros elsewhere); one CTA
// per row.
__global__ void k_csr_to_dense(int64_t n, int64_t ncols, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const double* __restrict__ val, double* __restrict__ D,
                               int64_t ld) {
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
    double* row = D + r * ld;
    for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) row[c] = 0.0;
    __syncthreads();
    for (int64_t k = rowptr[r] + threadIdx.x; k < rowptr[r + 1]; k += blockDim.x) row[col[k]] = val[k];
    __syncthreads();
  }
}
int launch_csr_to_dense(pase_ctx* h, int64_t n, int64_t ncols, const int64_t* rowptr, const int32_t* col,
                        const double* val, double* D, int64_t ld) {
  if (n == 0) return PASE_OK;
  k_csr_to_dense<<<(unsigned)std::min<int64_t>(n, 152 * 8), 256, 0, h->stream>>>(n, ncols, rowptr, col, val, D, ld);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// B[j][i] = A[i][j] for an rows x cols block
__global__ void k_transpose(int64_t rows, int64_t cols, const double* __restrict__ A, int64_t lda,
                            double* __restrict__ B, int64_t ldb) {
  const int64_t total = rows * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / cols, j = idx % cols;
    B[j * ldb + i] = A[i * lda + j];
  }
}
int launch_transpose(pase_ctx* h, int64_t rows, int64_t cols, const double* A, int64_t lda, double* B, int64_t ldb) {
  const int64_t total = rows * cols;
  if (total == 0) return PASE_OK;
  k_transpose<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, h->stream>>>(rows, cols, A, lda,
                                                                                                 B, ldb);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// dst[r][c] = src[r][idx[c]] for r < n, c < k
__global__ void k_gather_cols(int64_t n, int k, const double* __restrict__ src, int64_t lds,
                              const int* __restrict__ idx, double* __restrict__ dst, int64_t ldd) {
  const int64_t total = n * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int c = (int)(t % k);
    dst[r * ldd + c] = src[r * lds + idx[c]];
  }
}
int launch_gather_cols(pase_ctx* h, int64_t n, int k, const double* src, int64_t lds, const int* idx, double* dst,
                       int64_t ldd) {
  const int64_t total = n * k;
  if (total == 0) return PASE_OK;
  k_gather_cols<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, h->stream>>>(n, k, src, lds, idx,
                                                                                                   dst, ldd);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

}  // namespace pase
