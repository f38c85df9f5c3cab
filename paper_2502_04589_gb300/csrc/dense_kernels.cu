// Dense kernels: tall-skinny Gram products X^T Y and block updates X C over many rows
// (the alpha/beta blocks and the prolongation of Alg. 3 steps 4 and 6, and the block
// operations of the step-(c) eigensolver), the dense coarse-grid multiply, and small
// single-CTA dense routines (symmetric-definite eigensolver, Cholesky solve, GEMM).
//
// FP64 on this part runs at ~1.2 TFLOP/s against ~75 TFLOP/s FP32, so the FP64 kernels
// are ALU-bound: they are laid out to keep the FP64 pipe busy (register tiles fed from
// shared memory) rather than to minimise bytes.
#include <float.h>

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
  static bool attr_set = false;
  if (!attr_set) {
    PASE_CUDA(cudaFuncSetAttribute(k_ts_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
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
  static bool attr_set = false;
  if (!attr_set) {
    PASE_CUDA(cudaFuncSetAttribute(k_ts_gemm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
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
  // red: >= 32 doubles of shared memory
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < nw; ++w) s += red[w];
    red[32] = s;
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
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s = fmax(s, red[w]);
    red[32] = s;
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
// The k smallest pairs of GA c = lambda GB c (n x n symmetric, GB positive definite), one
// CTA, FP64.  Steps: diagonal scaling D = diag(GB)^-1/2; Cholesky D GB D = L L^T;
// K = L^-1 (D GA D) L^-T; Householder tridiagonalisation Q^T K Q = T; eigenvalues of T by
// bisection on Sturm counts; eigenvectors of T by inverse iteration (vectors of one
// cluster re-orthogonalised against each other); back-transform c = D L^-T Q z.
// Output C (n x k, ldc) is GB-orthonormal.  Directions of a numerically dependent basis
// (scaled Cholesky pivot below kPivTol) are dropped; status[0] = 1 only if fewer than k
// directions remain.
constexpr double kPivTol = 1e-10;
constexpr int kClusterRR = 16;

__device__ int sturm_count(int n, const double* d, const double* e, double x) {
  // number of eigenvalues of T strictly below x
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    if (q == 0.0) q = -DBL_MIN * 1e8;
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (q < 0) ++cnt;
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

// Solve (T - lam I) x = b in place (b -> x), tridiagonal LU with partial pivoting.
// Work arrays l, u0, u1, u2, piv of length n.
__device__ void tri_solve(int n, const double* d, const double* e, double lam, double* b,
                          double* u0, double* u1, double* u2, int* piv, double tiny) {
  // rows: main diag a_i = d_i - lam, sub/super e_i
  for (int i = 0; i < n; ++i) {
    u0[i] = d[i] - lam;
    u1[i] = (i < n - 1) ? e[i] : 0.0;
    u2[i] = 0.0;
  }
  // forward elimination with row swaps (u0 diag, u1 first super, u2 second super)
  for (int i = 0; i < n - 1; ++i) {
    const double sub = e[i];  // element (i+1, i)
    if (fabs(u0[i]) >= fabs(sub)) {
      piv[i] = 0;
      if (u0[i] == 0.0) u0[i] = tiny;
      const double f = sub / u0[i];
      u0[i + 1] -= f * u1[i];
      // u2[i] stays 0
      b[i + 1] -= f * b[i];
      u2[i] = 0.0;
      // store multiplier implicitly (not needed: b updated on the fly)
    } else {
      piv[i] = 1;
      const double f = u0[i] / sub;
      // swap rows i and i+1
      const double r0 = sub, r1 = u0[i + 1], r2 = (i + 1 < n - 1) ? e[i + 1] : 0.0;
      const double o1 = u1[i];
      u0[i] = r0;
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
  // back substitution
  b[n - 1] /= u0[n - 1];
  if (n >= 2) {
    b[n - 2] = (b[n - 2] - u1[n - 2] * b[n - 1]) / u0[n - 2];
    for (int i = n - 3; i >= 0; --i) b[i] = (b[i] - u1[i] * b[i + 1] - u2[i] * b[i + 2]) / u0[i];
  }
}

__global__ void __launch_bounds__(1024) k_sygv(int n, int k, const double* __restrict__ GA, int lda,
                                               const double* __restrict__ GB, int ldb, double* work,
                                               double* __restrict__ lam, double* __restrict__ C,
                                               int ldc, int* status) {
  __shared__ double red[40];
  __shared__ int s_fail;
  __shared__ double s_lo, s_hi;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* K = work;                // n*n  (becomes tridiagonal + Householder vectors)
  double* L = K + (int64_t)n * n;  // n*n
  double* Z = L + (int64_t)n * n;  // n*k
  double* d = Z + (int64_t)n * k;  // n
  double* e = d + n;               // n
  double* tau = e + n;             // n
  double* sc = tau + n;            // n
  double* v = sc + n;              // n
  double* p = v + n;               // n
  double* iw = p + n;              // 4 n k  (inverse iteration scratch)
  int* ipiv = reinterpret_cast<int*>(iw + (int64_t)4 * n * k);  // n k
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // 1. scaling; a zero column (a locked search direction) gets scale 0 and is dropped
  for (int i = tid; i < n; i += nt) {
    const double g = GB[(int64_t)i * ldb + i];
    if (!(g >= 0.0) || !isfinite(g)) s_fail = 1;
    sc[i] = (g > 0.0) ? rsqrt(g) : 0.0;
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) status[0] = 1;
    return;
  }
  for (int64_t idx = tid; idx < (int64_t)n * n; idx += nt) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    const double s = sc[i] * sc[j];
    K[idx] = s * 0.5 * (GA[(int64_t)i * lda + j] + GA[(int64_t)j * lda + i]);
    L[idx] = s * 0.5 * (GB[(int64_t)i * ldb + j] + GB[(int64_t)j * ldb + i]);
  }
  __syncthreads();
  // 2. Cholesky (lower, in place in L) with dropping: a pivot below kPivTol (relative to
  //    the unit diagonal after scaling) marks a direction numerically dependent on the
  //    earlier ones; its column is zeroed, L[j][j] = 1, and the direction is later given an
  //    eigenvalue above the whole spectrum so that no returned vector uses it.
  __shared__ int s_drop;
  if (tid == 0) s_drop = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double dj = L[(int64_t)j * n + j];
    const bool drop = !(dj > kPivTol) || !isfinite(dj);
    __syncthreads();
    if (tid == 0) {
      L[(int64_t)j * n + j] = drop ? 1.0 : sqrt(dj);
      if (drop) {
        ++s_drop;
        tau[j] = 1.0;  // tau doubles as the drop mask until step 4
      } else {
        tau[j] = 0.0;
      }
    }
    __syncthreads();
    const double ljj = L[(int64_t)j * n + j];
    for (int i = j + 1 + tid; i < n; i += nt) L[(int64_t)i * n + j] = drop ? 0.0 : L[(int64_t)i * n + j] / ljj;
    __syncthreads();
    if (!drop) {
      const int len = n - j - 1;
      for (int idx = tid; idx < len * len; idx += nt) {
        const int i = j + 1 + idx / len, l = j + 1 + idx % len;
        if (l <= i) L[(int64_t)i * n + l] -= L[(int64_t)i * n + j] * L[(int64_t)l * n + j];
      }
    }
    __syncthreads();
  }
  if (n - s_drop < k) {
    if (tid == 0) status[0] = 1;
    return;
  }
  // 3. K <- L^-1 K  (row i after rows < i; parallel over columns)
  for (int i = 0; i < n; ++i) {
    const double lii = L[(int64_t)i * n + i];
    for (int c = tid; c < n; c += nt) {
      double s = K[(int64_t)i * n + c];
      for (int l = 0; l < i; ++l) s -= L[(int64_t)i * n + l] * K[(int64_t)l * n + c];
      K[(int64_t)i * n + c] = s / lii;
    }
    __syncthreads();
  }
  //    K <- K L^-T  (column i after columns < i; parallel over rows)
  for (int i = 0; i < n; ++i) {
    const double lii = L[(int64_t)i * n + i];
    for (int r = tid; r < n; r += nt) {
      double s = K[(int64_t)r * n + i];
      for (int l = 0; l < i; ++l) s -= K[(int64_t)r * n + l] * L[(int64_t)i * n + l];
      K[(int64_t)r * n + i] = s / lii;
    }
    __syncthreads();
  }
  for (int64_t idx = tid; idx < (int64_t)n * n; idx += nt) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (i < j) {
      const double a = 0.5 * (K[(int64_t)i * n + j] + K[(int64_t)j * n + i]);
      K[(int64_t)i * n + j] = a;
      K[(int64_t)j * n + i] = a;
    }
  }
  __syncthreads();
  if (s_drop > 0) {
    // dropped directions get an eigenvalue just above the kept spectrum (Gershgorin
    // bound of the kept rows), so they are never among the k smallest and do not
    // inflate the norm that scales the inverse-iteration tolerances
    double part = 0.0;
    for (int i = tid; i < n; i += nt) {
      if (tau[i] != 0.0) continue;
      double r = 0.0;
      for (int j = 0; j < n; ++j)
        if (tau[j] == 0.0) r += fabs(K[(int64_t)i * n + j]);
      part = fmax(part, r);
    }
    const double big = 2.0 * block_max(part, red) + 1.0;
    for (int64_t idx = tid; idx < (int64_t)n * n; idx += nt) {
      const int i = (int)(idx / n), j = (int)(idx % n);
      if (tau[i] != 0.0 || tau[j] != 0.0) K[idx] = (i == j) ? big : 0.0;
    }
    __syncthreads();
  }
  // 4. Householder tridiagonalisation; reflector j acts on rows/cols j+1..n-1 and its
  //    vector (v[0] = 1 implicit) is kept in K[(j+1..n-1)*n + j], tau[j].
  for (int j = 0; j + 2 < n; ++j) {
    const int len = n - j - 1;
    double* A22 = K + (int64_t)(j + 1) * n + (j + 1);
    // norm of x = K[j+1.., j]
    double part = 0.0;
    for (int r = 1 + tid; r < len; r += nt) {
      const double x = K[(int64_t)(j + 1 + r) * n + j];
      part += x * x;
    }
    const double sig = block_sum(part, red);
    const double x0 = K[(int64_t)(j + 1) * n + j];
    double beta, t;
    if (sig == 0.0) {
      t = 0.0;
      beta = x0;
    } else {
      const double nrm = sqrt(x0 * x0 + sig);
      beta = (x0 >= 0.0) ? -nrm : nrm;
      t = (beta - x0) / beta;
    }
    const double scal = (sig == 0.0) ? 0.0 : 1.0 / (x0 - beta);
    for (int r = tid; r < len; r += nt) v[r] = (r == 0) ? 1.0 : K[(int64_t)(j + 1 + r) * n + j] * scal;
    __syncthreads();
    if (t != 0.0) {
      // p = t A22 v
      for (int r = tid; r < len; r += nt) {
        double s = 0.0;
        const double* row = A22 + (int64_t)r * n;
        for (int c = 0; c < len; ++c) s = fma(row[c], v[c], s);
        p[r] = t * s;
      }
      __syncthreads();
      double pv = 0.0;
      for (int r = tid; r < len; r += nt) pv += p[r] * v[r];
      const double Kc = 0.5 * t * block_sum(pv, red);
      for (int r = tid; r < len; r += nt) p[r] -= Kc * v[r];
      __syncthreads();
      for (int64_t idx = tid; idx < (int64_t)len * len; idx += nt) {
        const int r = (int)(idx / len), c = (int)(idx % len);
        A22[(int64_t)r * n + c] -= v[r] * p[c] + p[r] * v[c];
      }
    }
    __syncthreads();
    if (tid == 0) {
      d[j] = K[(int64_t)j * n + j];
      e[j] = beta;
      tau[j] = t;
    }
    for (int r = 1 + tid; r < len; r += nt) K[(int64_t)(j + 1 + r) * n + j] = v[r];
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = K[(int64_t)(n - 2) * n + (n - 2)];
      e[n - 2] = K[(int64_t)(n - 1) * n + (n - 2)];
      tau[n - 2] = 0.0;
    }
    d[n - 1] = K[(int64_t)(n - 1) * n + (n - 1)];
    e[n - 1] = 0.0;
    // Gershgorin interval
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
    }
    const double pad = 1e-14 * fmax(fabs(lo), fabs(hi)) + DBL_MIN;
    s_lo = lo - pad;
    s_hi = hi + pad;
  }
  __syncthreads();
  const double tnorm = fmax(fabs(s_lo), fabs(s_hi));
  // 5. bisection: lam[i] = i-th smallest (0-based)
  for (int i = tid; i < k; i += nt) {
    double a = s_lo, b = s_hi;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a + b);
      if (mid <= a || mid >= b) break;
      if (b - a <= 2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b))) break;
      if (sturm_count(n, d, e, mid) > i) b = mid;
      else a = mid;
    }
    lam[i] = 0.5 * (a + b);
  }
  __syncthreads();
  // 6. inverse iteration.  Eigenvalues closer than ctol = 1e-6 |T| form a cluster, owned by
  //    the thread of its first member: its vectors are re-orthogonalised against each
  //    other (vectors of close eigenvalues computed independently lose orthogonality by
  //    ~eps |T| / gap) and then rotated by a Rayleigh-Ritz step inside the cluster, so
  //    that every returned pair has value = Rayleigh quotient of its vector.
  const double ctol = 1e-6 * tnorm;
  const double tiny = DBL_EPSILON * tnorm + DBL_MIN;
  for (int i = tid; i < k; i += nt) {
    if (i > 0 && lam[i] - lam[i - 1] <= ctol) continue;  // not a cluster head
    int last = i;
    while (last + 1 < k && lam[last + 1] - lam[last] <= ctol) ++last;
    double* u0 = iw + (int64_t)4 * n * i;
    double* u1 = u0 + n;
    double* u2 = u1 + n;
    double* bb = u2 + n;
    int* pv_ = ipiv + (int64_t)n * i;
    for (int q = i; q <= last; ++q) {
      double* z = Z + q;  // column q, stride k
      for (int r = 0; r < n; ++r) bb[r] = hash_unit((unsigned)q, (unsigned)r) + 1e-3;
      for (int it = 0; it < 3; ++it) {
        tri_solve(n, d, e, lam[q], bb, u0, u1, u2, pv_, tiny);
        for (int pass = 0; pass < 2; ++pass)
          for (int o = i; o < q; ++o) {
            double dot = 0.0;
            for (int r = 0; r < n; ++r) dot += bb[r] * Z[(int64_t)r * k + o];
            for (int r = 0; r < n; ++r) bb[r] -= dot * Z[(int64_t)r * k + o];
          }
        double nrm = 0.0;
        for (int r = 0; r < n; ++r) nrm += bb[r] * bb[r];
        nrm = sqrt(nrm);
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int r = 0; r < n; ++r) bb[r] *= inv;
      }
      for (int r = 0; r < n; ++r) z[(int64_t)r * k] = bb[r];
    }
    const int s = last - i + 1;
    if (s >= 2 && s <= kClusterRR) {
      // H = Q^T T Q for the cluster block Q = Z[:, i..last], then cyclic Jacobi on H
      double H[kClusterRR * kClusterRR];
      for (int a = 0; a < s; ++a)
        for (int b = a; b < s; ++b) {
          double acc = 0.0;
          for (int r = 0; r < n; ++r) {
            double tq = d[r] * Z[(int64_t)r * k + i + b];
            if (r > 0) tq += e[r - 1] * Z[(int64_t)(r - 1) * k + i + b];
            if (r < n - 1) tq += e[r] * Z[(int64_t)(r + 1) * k + i + b];
            acc += Z[(int64_t)r * k + i + a] * tq;
          }
          H[a * s + b] = acc;
          H[b * s + a] = acc;
        }
      for (int sweep = 0; sweep < 12; ++sweep) {
        double off = 0.0;
        for (int a = 0; a < s; ++a)
          for (int b = a + 1; b < s; ++b) off += H[a * s + b] * H[a * s + b];
        if (off <= 1e-32 * (tnorm * tnorm)) break;
        for (int a = 0; a < s; ++a)
          for (int b = a + 1; b < s; ++b) {
            const double hab = H[a * s + b];
            if (hab == 0.0) continue;
            const double th = 0.5 * (H[b * s + b] - H[a * s + a]) / hab;
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
            for (int l = 0; l < s; ++l) {  // columns a, b of H
              const double ha = H[l * s + a], hb = H[l * s + b];
              H[l * s + a] = c * ha - sn * hb;
              H[l * s + b] = sn * ha + c * hb;
            }
            for (int l = 0; l < s; ++l) {  // rows a, b
              const double ha = H[a * s + l], hb = H[b * s + l];
              H[a * s + l] = c * ha - sn * hb;
              H[b * s + l] = sn * ha + c * hb;
            }
            for (int r = 0; r < n; ++r) {  // vectors
              const double za = Z[(int64_t)r * k + i + a], zb = Z[(int64_t)r * k + i + b];
              Z[(int64_t)r * k + i + a] = c * za - sn * zb;
              Z[(int64_t)r * k + i + b] = sn * za + c * zb;
            }
          }
      }
      // sort the cluster ascending by its Rayleigh quotients
      for (int a = 0; a < s; ++a) {
        int best = a;
        for (int b = a + 1; b < s; ++b)
          if (H[b * s + b] < H[best * s + best]) best = b;
        if (best != a) {
          const double t = H[a * s + a];
          H[a * s + a] = H[best * s + best];
          H[best * s + best] = t;
          for (int r = 0; r < n; ++r) {
            const double za = Z[(int64_t)r * k + i + a];
            Z[(int64_t)r * k + i + a] = Z[(int64_t)r * k + i + best];
            Z[(int64_t)r * k + i + best] = za;
          }
        }
        lam[i + a] = H[a * s + a];
      }
    }
  }
  __syncthreads();
  // 7. back-transform z <- H_0 ... H_{n-3} z, reflector j acting on rows j+1..
  for (int j = n - 3; j >= 0; --j) {
    const double t = tau[j];
    if (t == 0.0) continue;
    const int len = n - j - 1;
    for (int c = tid; c < k; c += nt) {
      double s = Z[(int64_t)(j + 1) * k + c];
      for (int r = 1; r < len; ++r) s = fma(K[(int64_t)(j + 1 + r) * n + j], Z[(int64_t)(j + 1 + r) * k + c], s);
      s *= t;
      Z[(int64_t)(j + 1) * k + c] -= s;
      for (int r = 1; r < len; ++r) Z[(int64_t)(j + 1 + r) * k + c] -= s * K[(int64_t)(j + 1 + r) * n + j];
    }
    __syncthreads();
  }
  //    c = D L^-T z  (back substitution, parallel over columns)
  for (int c = tid; c < k; c += nt) {
    for (int i = n - 1; i >= 0; --i) {
      double s = Z[(int64_t)i * k + c];
      for (int l = i + 1; l < n; ++l) s -= L[(int64_t)l * n + i] * Z[(int64_t)l * k + c];
      Z[(int64_t)i * k + c] = s / L[(int64_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) C[(int64_t)i * ldc + c] = sc[i] * Z[(int64_t)i * k + c];
  }
  if (tid == 0) status[0] = 0;
}

size_t small_sygv_work_doubles(int n, int k) {
  return (size_t)2 * n * n + (size_t)n * k + 6 * (size_t)n + (size_t)4 * n * k + (size_t)n * k;  // ints fit
}

int small_sygv(pase_ctx* h, int n, int k, const double* GA, int lda, const double* GB, int ldb,
               double* lam, double* C, int ldc, int* status_dev) {
  if (n <= 0 || k <= 0 || k > n) return fail(PASE_ERR_INVALID_ARG, "small_sygv: bad size");
  if (small_sygv_work_doubles(n, k) > h->w.eigwork_doubles)
    return fail(PASE_ERR_INVALID_ARG, "small_sygv: workspace too small");
  k_sygv<<<1, 1024, 0, h->stream>>>(n, k, GA, lda, GB, ldb, h->w.eigwork, lam, C, ldc, status_dev);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

}  // namespace pase
