// Sparse-matrix x multivector kernels (CSR, node-major multivectors [n][m]).
//
// One kernel template covers every sparse product on the path: the fused A_h/M_h
// product of the projection step (Alg. 3 step 4: A_h W and B_h W share one sparsity
// pattern, so one pass over the index stream serves both), the eigen-residual
// M U Lambda - A U with its column norms (the convergence test of §6), the damped
// Jacobi sweep and residual of the multigrid solve, restriction P^T and prolongation P.
//
// Layout: thread group of tpr = m / VW threads per row, VW = 16 bytes / sizeof(T), so
// each thread owns one 16-byte column slice and every X row is read as tpr contiguous
// 16-byte loads; the tpr threads of a row read the same index/value (broadcast).
// In FP64 these kernels are bound by the FP64 pipe (1.2 TFLOP/s on this part), in FP32
// by HBM / L2 bandwidth.
#include "pase_internal.h"

namespace pase {

template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
  static constexpr int W = 2;
  __device__ static inline void load(const double* p, double (&v)[2]) {
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  }
  __device__ static inline void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};
template <>
struct Vec16<float> {
  static constexpr int W = 4;
  __device__ static inline void load(const float* p, float (&v)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
  __device__ static inline void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_csr(int64_t n, int m, int64_t ldx, int64_t ldy, int tpr, int rpb,
                                             const int64_t* __restrict__ rowptr,
                                             const int32_t* __restrict__ col,
                                             const T* __restrict__ va, const T* __restrict__ vm,
                                             const T* __restrict__ X, const T* __restrict__ X2,
                                             const T* __restrict__ B, const T* __restrict__ dinv,
                                             const double* __restrict__ lam, T omega,
                                             T* __restrict__ Y1, T* __restrict__ Y2,
                                             double* __restrict__ partial) {
  using V = Vec16<T>;
  constexpr int VW = V::W;
  const int tx = threadIdx.x % tpr;
  const int ty = threadIdx.x / tpr;
  const bool active = ty < rpb;
  const int c0 = tx * VW;
  double sr[VW], sm[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) sr[v] = sm[v] = 0.0;
  double lv[VW];
  if (MODE == CSR_EIGRES) {
#pragma unroll
    for (int v = 0; v < VW; ++v) lv[v] = active ? lam[c0 + v] : 0.0;
  }
  if (active) {
    for (int64_t row = (int64_t)blockIdx.x * rpb + ty; row < n; row += (int64_t)gridDim.x * rpb) {
      T a1[VW], a2[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) a1[v] = a2[v] = T(0);
      const int64_t k0 = rowptr[row], k1 = rowptr[row + 1];
      for (int64_t k = k0; k < k1; ++k) {
        const int64_t c = col[k];
        const T a = va[k];
        T x[VW];
        V::load(X + c * ldx + c0, x);
#pragma unroll
        for (int v = 0; v < VW; ++v) a1[v] = fma(a, x[v], a1[v]);
        if (MODE == CSR_MV_AM || MODE == CSR_EIGRES) {
          const T b = vm[k];
#pragma unroll
          for (int v = 0; v < VW; ++v) a2[v] = fma(b, x[v], a2[v]);
        }
        if (MODE == CSR_MV2) {
          T x2[VW];
          V::load(X2 + c * ldx + c0, x2);
#pragma unroll
          for (int v = 0; v < VW; ++v) a2[v] = fma(a, x2[v], a2[v]);
        }
      }
      const int64_t o = row * ldy + c0;
      const int64_t ox = row * ldx + c0;
      if (MODE == CSR_MV) {
        V::store(Y1 + o, a1);
      } else if (MODE == CSR_MVDOT) {
        V::store(Y1 + o, a1);
        T x[VW];
        V::load(X + ox, x);
#pragma unroll
        for (int v = 0; v < VW; ++v) sr[v] = fma((double)x[v], (double)a1[v], sr[v]);
      } else if (MODE == CSR_MV_AM || MODE == CSR_MV2) {
        V::store(Y1 + o, a1);
        V::store(Y2 + o, a2);
      } else if (MODE == CSR_RESID || MODE == CSR_ADD) {
        T b[VW];
        V::load(B + o, b);
#pragma unroll
        for (int v = 0; v < VW; ++v) a1[v] = (MODE == CSR_RESID) ? b[v] - a1[v] : b[v] + a1[v];
        V::store(Y1 + o, a1);
      } else if (MODE == CSR_JACOBI) {
        T b[VW], x[VW];
        V::load(B + o, b);
        V::load(X + ox, x);
        const T d = omega * dinv[row];
#pragma unroll
        for (int v = 0; v < VW; ++v) a1[v] = fma(d, b[v] - a1[v], x[v]);
        V::store(Y1 + o, a1);
      } else if (MODE == CSR_EIGRES) {
        T r[VW];
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          r[v] = (T)fma((double)a2[v], lv[v], -(double)a1[v]);
          sr[v] = fma((double)r[v], (double)r[v], sr[v]);
          sm[v] = fma((double)a2[v], (double)a2[v], sm[v]);
        }
        if (Y1) V::store(Y1 + o, r);
      }
    }
  }
  if (MODE == CSR_EIGRES || MODE == CSR_MVDOT) {
    // block reduction of the column sums: red[nsum][rpb][m] with rpb*m <= 512*VW;
    // EIGRES keeps two sums per column (|r|^2, |Mx|^2), MVDOT one (x . Ax)
    constexpr int nsum = (MODE == CSR_EIGRES) ? 2 : 1;
    __shared__ double red[nsum * 512 * VW];
    if (active) {
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        red[ty * m + c0 + v] = sr[v];
        if (nsum == 2) red[(nsum - 1) * rpb * m + ty * m + c0 + v] = sm[v];
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nsum * m; j += blockDim.x) {
      const int half = j / m, c = j % m;
      double s = 0.0;
      for (int r = 0; r < rpb; ++r) s += red[half * rpb * m + r * m + c];
      partial[(int64_t)blockIdx.x * nsum * m + j] = s;
    }
  }
}

static inline int grid_for(int64_t n, int rpb, int cap) {
  int64_t g = (n + rpb - 1) / rpb;
  if (g < 1) g = 1;
  if (cap > 0 && g > cap) g = cap;
  if (g > 0x7fffffffLL) g = 0x7fffffff;
  return (int)g;
}


template <typename T>
int launch_csr(pase_ctx* h, int mode, int m, const DevCSR& A, const T* va, const T* vm,
               const T* X, const T* X2, const T* B, const T* dinv, const double* lam,
               double omega, T* Y1, T* Y2, double* partial, int* nblocks_out, int64_t ldx,
               int64_t ldy) {
  if (ldx <= 0) ldx = m;
  if (ldy <= 0) ldy = m;
  constexpr int VW = 16 / sizeof(T);
  if (m % 8 != 0 || m <= 0 || m / VW > 512) return fail(PASE_ERR_INVALID_ARG, "launch_csr: bad m");
  const int tpr = m / VW;
  int bs = A.block > 0 ? A.block : 256;
  if (bs < tpr) bs = ((tpr + 31) / 32) * 32;
  if (bs > 512) bs = 512;
  const int rpb = bs / tpr;
  const int grid = grid_for(A.nrows, rpb, (mode == CSR_EIGRES || mode == CSR_MVDOT) ? kReduceBlocksHost : 0);
  if (nblocks_out) *nblocks_out = grid;
  if (A.nrows == 0) return PASE_OK;
  auto s = h->stream;
  const T om = (T)omega;
  int prof_id = -1;
  if (h->prof_kernel >= 0 && !h->lv.empty() && A.rowptr == h->lv[0].A.rowptr) {
    if (mode == CSR_MV_AM && sizeof(T) == 8) prof_id = PASE_KERNEL_SPMM_AM_FP64;
    if (mode == CSR_JACOBI) prof_id = sizeof(T) == 8 ? PASE_KERNEL_JACOBI_FP64 : PASE_KERNEL_JACOBI_FP32;
  }
  if (sizeof(T) == 4 && h->opt.stencil && A.st_use && h->tc_err && stencil_ok(A, mode, m, ldx, ldy, omega)) {
    // grid-neighbour operator: the structured FP32 kernel (no column indices, X reuse in registers)
    prof_begin(h, prof_id);
    const int rc = launch_stencil(h, mode, m, A, (const float*)X, (const float*)B, omega, (float*)Y1);
    prof_end(h, prof_id);
    return rc;
  }
  prof_begin(h, prof_id);
#define PASE_CSR_CASE(MD)                                                                   \
  case MD:                                                                                  \
    k_csr<T, MD><<<grid, bs, 0, s>>>(A.nrows, m, ldx, ldy, tpr, rpb, A.rowptr, A.col, va, vm, X, X2, \
                                       B, dinv, lam, om, Y1, Y2, partial);                   \
    break;
  switch (mode) {
    PASE_CSR_CASE(CSR_MV)
    PASE_CSR_CASE(CSR_MV_AM)
    PASE_CSR_CASE(CSR_RESID)
    PASE_CSR_CASE(CSR_JACOBI)
    PASE_CSR_CASE(CSR_EIGRES)
    PASE_CSR_CASE(CSR_MV2)
    PASE_CSR_CASE(CSR_ADD)
    PASE_CSR_CASE(CSR_MVDOT)
    default:
      return fail(PASE_ERR_INVALID_ARG, "launch_csr: bad mode");
  }
#undef PASE_CSR_CASE
  prof_end(h, prof_id);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

template int launch_csr<double>(pase_ctx*, int, int, const DevCSR&, const double*, const double*,
                                const double*, const double*, const double*, const double*,
                                const double*, double, double*, double*, double*, int*, int64_t,
                                int64_t);
template int launch_csr<float>(pase_ctx*, int, int, const DevCSR&, const float*, const float*,
                               const float*, const float*, const float*, const float*,
                               const double*, double, float*, float*, double*, int*, int64_t,
                               int64_t);

// ------------------------------------------------------------------ elementwise kernels

template <typename T>
__global__ void k_scale_dinv(int64_t n, int m, const T* __restrict__ dinv, T omega,
                             const T* __restrict__ B, T* __restrict__ Y) {
  const int64_t total = n * m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    Y[i] = omega * dinv[i / m] * B[i];
}

static inline int ew_grid(int64_t count) {
  int64_t g = (count + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
int launch_scale_dinv(pase_ctx* h, int64_t n, int m, const T* dinv, double omega, const T* B,
                      T* Y) {
  k_scale_dinv<T><<<ew_grid(n * m), 256, 0, h->stream>>>(n, m, dinv, (T)omega, B, Y);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}
template int launch_scale_dinv<double>(pase_ctx*, int64_t, int, const double*, double,
                                       const double*, double*);
template int launch_scale_dinv<float>(pase_ctx*, int64_t, int, const float*, double, const float*,
                                      float*);

__global__ void k_axpy(int64_t count, double a, const double* __restrict__ x,
                       const double* __restrict__ y, double* __restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] = fma(a, x[i], y[i]);
}
int launch_axpy(pase_ctx* h, int64_t count, double a, const double* x, const double* y,
                double* z) {
  k_axpy<<<ew_grid(count), 256, 0, h->stream>>>(count, a, x, y, z);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

__global__ void k_f64_to_f32(int64_t count, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
int launch_f64_to_f32(pase_ctx* h, int64_t count, const double* x, float* y) {
  k_f64_to_f32<<<ew_grid(count), 256, 0, h->stream>>>(count, x, y);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

__global__ void k_add_f32_to_f64(int64_t count, const double* __restrict__ u,
                                 const float* __restrict__ e, double* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = u[i] + (double)e[i];
}
int launch_add_f32_to_f64(pase_ctx* h, int64_t count, const double* u, const float* e,
                          double* w) {
  k_add_f32_to_f64<<<ew_grid(count), 256, 0, h->stream>>>(count, u, e, w);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

__global__ void k_copy_cols(int64_t n, int k, const double* __restrict__ src, int lds,
                            double* __restrict__ dst, int ldd) {
  const int64_t total = n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / k;
    const int c = (int)(i % k);
    dst[r * ldd + c] = src[r * lds + c];
  }
}
int launch_copy_cols(pase_ctx* h, int64_t n, int k, const double* src, int lds, double* dst,
                     int ldd) {
  if (n * k == 0) return PASE_OK;
  k_copy_cols<<<ew_grid(n * k), 256, 0, h->stream>>>(n, k, src, lds, dst, ldd);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

__global__ void k_fill(int64_t count, double v, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}
int launch_fill(pase_ctx* h, int64_t count, double v, double* x) {
  if (count == 0) return PASE_OK;
  k_fill<<<ew_grid(count), 256, 0, h->stream>>>(count, v, x);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// ------------------------------------------------------------------ CG building blocks
// Column inner products out[j] = sum_i X[i][j] Y[i][j] of two [n][m] blocks: tpr = m/2
// threads per row (one 16-byte column pair each), a grid-stride loop over rows, a fixed
// per-block tree into partial[block][m] and the deterministic cross-block reduction.
__global__ void __launch_bounds__(256) k_coldot(int64_t n, int m, int tpr, int rpb, const double* __restrict__ X,
                                                const double* __restrict__ Y, double* __restrict__ partial) {
  const int tx = threadIdx.x % tpr, ty = threadIdx.x / tpr;
  const bool active = ty < rpb;
  const int c0 = 2 * tx;
  double s0 = 0.0, s1 = 0.0;
  if (active)
    for (int64_t row = (int64_t)blockIdx.x * rpb + ty; row < n; row += (int64_t)gridDim.x * rpb) {
      const double2 x = __ldg(reinterpret_cast<const double2*>(X + row * m + c0));
      const double2 y = __ldg(reinterpret_cast<const double2*>(Y + row * m + c0));
      s0 = fma(x.x, y.x, s0);
      s1 = fma(x.y, y.y, s1);
    }
  __shared__ double red[512];  // rpb * m = (256 / tpr) * 2 tpr <= 512
  if (active) {
    red[ty * m + c0] = s0;
    red[ty * m + c0 + 1] = s1;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += red[r * m + j];
    partial[(int64_t)blockIdx.x * m + j] = s;
  }
}

// out[j] = num[j] / den[j] if den[j] > 0, else 0 (a column whose CG has broken down or
// converged exactly stops moving)
__global__ void k_ratio(int m, const double* __restrict__ num, const double* __restrict__ den,
                        double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) out[j] = den[j] > 0.0 ? num[j] / den[j] : 0.0;
}

// X += P diag(alpha), R -= Q diag(alpha), one 16-byte column pair per thread
__global__ void k_cg_update(int64_t pairs, int m, const double* __restrict__ alpha, const double* __restrict__ P,
                            const double* __restrict__ Q, double* __restrict__ X, double* __restrict__ R) {
  const int hm = m / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pairs; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = 2 * (int)(i % hm);
    const double a0 = alpha[c], a1 = alpha[c + 1];
    const double2 p = __ldg(reinterpret_cast<const double2*>(P) + i);
    const double2 q = __ldg(reinterpret_cast<const double2*>(Q) + i);
    double2 x = reinterpret_cast<double2*>(X)[i];
    double2 r = reinterpret_cast<double2*>(R)[i];
    x.x = fma(a0, p.x, x.x);
    x.y = fma(a1, p.y, x.y);
    r.x = fma(-a0, q.x, r.x);
    r.y = fma(-a1, q.y, r.y);
    reinterpret_cast<double2*>(X)[i] = x;
    reinterpret_cast<double2*>(R)[i] = r;
  }
}

// P = Z + P diag(beta)
__global__ void k_cg_dir(int64_t pairs, int m, const double* __restrict__ beta, const double* __restrict__ Z,
                         double* __restrict__ P) {
  const int hm = m / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pairs; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = 2 * (int)(i % hm);
    const double2 z = __ldg(reinterpret_cast<const double2*>(Z) + i);
    double2 p = reinterpret_cast<double2*>(P)[i];
    p.x = fma(beta[c], p.x, z.x);
    p.y = fma(beta[c + 1], p.y, z.y);
    reinterpret_cast<double2*>(P)[i] = p;
  }
}

__global__ void k_f32_to_f64(int64_t count, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

int launch_coldot(pase_ctx* h, int64_t n, int m, const double* X, const double* Y, double* out) {
  if (m <= 0 || m % 2 != 0 || m > 512) return fail(PASE_ERR_INVALID_ARG, "coldot: bad m");
  if (n == 0) return launch_fill(h, m, 0.0, out);
  const int tpr = m / 2, rpb = 256 / tpr;
  const int grid = grid_for(n, rpb, kReduceBlocksHost);
  k_coldot<<<grid, 256, 0, h->stream>>>(n, m, tpr, rpb, X, Y, h->w.partial);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return launch_reduce_partials(h, grid, m, h->w.partial, out);
}

int launch_ratio(pase_ctx* h, int m, const double* num, const double* den, double* out) {
  k_ratio<<<(m + 127) / 128, 128, 0, h->stream>>>(m, num, den, out);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

int launch_cg_update(pase_ctx* h, int64_t n, int m, const double* alpha, const double* P, const double* Q,
                     double* X, double* R) {
  const int64_t pairs = n * (m / 2);
  if (pairs == 0) return PASE_OK;
  k_cg_update<<<ew_grid(pairs), 256, 0, h->stream>>>(pairs, m, alpha, P, Q, X, R);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

int launch_cg_dir(pase_ctx* h, int64_t n, int m, const double* beta, const double* Z, double* P) {
  const int64_t pairs = n * (m / 2);
  if (pairs == 0) return PASE_OK;
  k_cg_dir<<<ew_grid(pairs), 256, 0, h->stream>>>(pairs, m, beta, Z, P);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

int launch_f32_to_f64(pase_ctx* h, int64_t count, const float* x, double* y) {
  if (count == 0) return PASE_OK;
  k_f32_to_f64<<<ew_grid(count), 256, 0, h->stream>>>(count, x, y);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// out[j] = sum_b partial[b*width + j]; one block per output, deterministic tree.
__global__ void k_reduce_partials(int nblk, int width, const double* __restrict__ partial,
                                  double* __restrict__ out) {
  __shared__ double s[256];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partial[(int64_t)b * width + j];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = s[0];
}
int launch_reduce_partials(pase_ctx* h, int nblk, int width, const double* partial,
                           double* out) {
  if (width == 0) return PASE_OK;
  k_reduce_partials<<<width, 256, 0, h->stream>>>(nblk, width, partial, out);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// relres[j] = sqrt(|r_j|^2) / (|lambda_j| sqrt(|M u_j|^2)); norms = [|r|^2 (m), |Mu|^2 (m)]
__global__ void k_relres(int m, const double* __restrict__ norms, const double* __restrict__ lam,
                         double* __restrict__ relres) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) {
    const double den = fabs(lam[j]) * sqrt(norms[m + j]);
    relres[j] = den > 0.0 ? sqrt(norms[j]) / den : INFINITY;
  }
}
int launch_relres(pase_ctx* h, int m, const double* norms, const double* lam, double* relres) {
  k_relres<<<(m + 127) / 128, 128, 0, h->stream>>>(m, norms, lam, relres);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// C = a A + b B on a rows x cols strided block (C may alias A or B).
__global__ void k_geam(int64_t rows, int cols, double a, const double* A, int64_t lda, double b,
                       const double* B, int64_t ldb, double* C, int64_t ldc) {
  const int64_t total = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols;
    const int c = (int)(i % cols);
    const double va = (a != 0.0) ? a * A[r * lda + c] : 0.0;
    const double vb = (b != 0.0) ? b * B[r * ldb + c] : 0.0;
    C[r * ldc + c] = va + vb;
  }
}
int launch_geam(pase_ctx* h, int64_t rows, int cols, double a, const double* A, int64_t lda,
                double b, const double* B, int64_t ldb, double* C, int64_t ldc) {
  if (rows * cols == 0) return PASE_OK;
  k_geam<<<ew_grid(rows * cols), 256, 0, h->stream>>>(rows, cols, a, A, lda, b, B, ldb, C, ldc);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// X[r][c] = uniform(-0.5, 0.5) from a SplitMix64-style hash of (seed, r, c).
__global__ void k_hash_fill(int64_t rows, int cols, int64_t ld, unsigned seed, double* X) {
  const int64_t total = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols;
    const int c = (int)(i % cols);
    unsigned long long z = (unsigned long long)seed * 0x9E3779B97F4A7C15ULL + (unsigned long long)i + 1ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    X[r * ld + c] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}
int launch_hash_fill(pase_ctx* h, int64_t rows, int cols, int64_t ld, unsigned seed, double* X) {
  if (rows * cols == 0) return PASE_OK;
  k_hash_fill<<<ew_grid(rows * cols), 256, 0, h->stream>>>(rows, cols, ld, seed, X);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}
// rows row0..row0+k-1 of X (width k, stride ld) <- identity
__global__ void k_set_identity_rows(int64_t row0, int k, int64_t ld, double* X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k * k) X[(row0 + i / k) * ld + (i % k)] = (i / k == i % k) ? 1.0 : 0.0;
}
int launch_set_identity_rows(pase_ctx* h, int64_t row0, int k, int64_t ld, double* X) {
  k_set_identity_rows<<<(k * k + 255) / 256, 256, 0, h->stream>>>(row0, k, ld, X);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// Column j of X (rows 0..n-1, stride ld) is zeroed where crit[j] <= thresh.
__global__ void k_zero_cols_if(int64_t n, int m, int64_t ld, const double* __restrict__ crit,
                               double thresh, const double* __restrict__ thresh_dev, double* __restrict__ X) {
  if (thresh_dev) thresh = *thresh_dev;
  const int64_t total = n * m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % m);
    if (crit[c] <= thresh) X[(i / m) * ld + c] = 0.0;
  }
}
int launch_zero_cols_if(pase_ctx* h, int64_t n, int m, int64_t ld, const double* crit, double thresh,
                        double* X, const double* thresh_dev) {
  if (n * m == 0) return PASE_OK;
  k_zero_cols_if<<<ew_grid(n * m), 256, 0, h->stream>>>(n, m, ld, crit, thresh, thresh_dev, X);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// R = AX - BX diag(lam) over n rows of width m, with per-block column sums of |R|^2 and
// |BX|^2 in partial[b][2m] (the residual test of the step-(c) block eigensolver).
__global__ void __launch_bounds__(256) k_block_resid(int64_t n, int m, const double* __restrict__ AX,
                                                     const double* __restrict__ BX, int64_t ldin,
                                                     const double* __restrict__ lam,
                                                     double* __restrict__ R, int64_t ldr,
                                                     double* __restrict__ partial) {
  __shared__ double red[2 * 256];
  // thread -> column c, row group g
  const int c = threadIdx.x % m;
  const int g = threadIdx.x / m;
  const int groups = blockDim.x / m;
  double sr = 0.0, sb = 0.0;
  if (g < groups) {
    const double l = lam[c];
    for (int64_t r = (int64_t)blockIdx.x * groups + g; r < n; r += (int64_t)gridDim.x * groups) {
      const double b = BX[r * ldin + c];
      const double v = AX[r * ldin + c] - b * l;
      if (R) R[r * ldr + c] = v;
      sr = fma(v, v, sr);
      sb = fma(b, b, sb);
    }
  }
  red[threadIdx.x] = (g < groups) ? sr : 0.0;
  red[256 + threadIdx.x] = (g < groups) ? sb : 0.0;
  __syncthreads();
  if (threadIdx.x < m) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < groups; ++q) {
      a += red[q * m + threadIdx.x];
      b += red[256 + q * m + threadIdx.x];
    }
    partial[(int64_t)blockIdx.x * 2 * m + threadIdx.x] = a;
    partial[(int64_t)blockIdx.x * 2 * m + m + threadIdx.x] = b;
  }
}
int launch_block_resid(pase_ctx* h, int64_t n, int m, const double* AX, const double* BX,
                       int64_t ldin, const double* lam, double* R, int64_t ldr, int* nblk_out) {
  if (m > 256) return fail(PASE_ERR_INVALID_ARG, "block_resid: m > 256");
  const int groups = 256 / m;
  int64_t g = (n + groups - 1) / groups;
  if (g > kReduceBlocksHost) g = kReduceBlocksHost;
  if (g < 1) g = 1;
  *nblk_out = (int)g;
  k_block_resid<<<(int)g, 256, 0, h->stream>>>(n, m, AX, BX, ldin, lam, R, ldr, h->w.partial);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// ------------------------------------------------------------------ FP64 FMA rate
// Independent FMA chains (no memory traffic, the loop unrolled so that loop control does
// not share the issue slots): a measurement of the part's FP64 arithmetic rate.  Its eight
// dependent chains per thread reach about 85% of the nominal rate, below what the FP64
// Jacobi sweep sustains, so it is reported beside the nominal peak rather than used as one.
__global__ void __launch_bounds__(256) k_fma_fp64(int iters, double seed, double* out) {
  constexpr int kChains = 8;
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = seed * (threadIdx.x + 1 + j);
  const double b = 0.999999999, c = 1e-12;
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == -1.0) out[0] = s;  // never true; keeps the chains alive
}
int launch_fma_fp64(pase_ctx* h, double* out) {
  k_fma_fp64<<<kFmaBlocks, kFmaThreads, 0, h->stream>>>(kFmaIters, 1e-3, out);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

}  // namespace pase
