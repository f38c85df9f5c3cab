// The fused fine-level products of the projection (Alg. 3 step 4: A_h W, M_h W) and of
// the eigen-residual (M U Lambda - A U with its column norms, the §6 convergence test) in
// double-float arithmetic: every FP64 operand is carried as an unevaluated sum of two
// FP32 numbers (hi + lo, 48 significand bits) and the products and sums run on the FP32
// pipe with error-free transformations (Dekker's product through FMA, Knuth's two-sum).
//
// Why: on this part FP64 arithmetic is 1/62 of FP32, so the FP64 CSR kernel of these
// products is bound by the FP64 pipe (10 ms per fused product at the 128^3 bench workload
// against 0.57 ms of HBM traffic).  The double-float form keeps FP64-level accuracy (each
// product and sum exact to about 2^-48 relative to the row's sum of |a||x|) with about
// twelve FP32 operations per nonzero and column.
//
// Layout: the matrix values are split once at setup (hi = fl32(a), lo = fl32(a - hi));
// the multivector is split per call by k_split_df64 into two [N][m] FP32 blocks.  Values
// of magnitude above 2^100 would overflow the FP32 products, so the split raises a flag
// that the caller reports; values below 2^-100 lose relative, not absolute, accuracy.
#include "pase_internal.h"

namespace pase {

namespace {

constexpr int64_t kDfBigExp = 1023 + 100;  // biased exponent of 2^100

// (s, e) = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc += a * x, all three in double-float; the running sum's high part is kept exact by
// two-sum, the low part gathers the rounding errors and the cross terms
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float xh, float xl) {
  const float p = ah * xh;
  float e = fmaf(ah, xh, -p);  // exact error of the leading product
  e = fmaf(ah, xl, fmaf(al, xh, e));
  float s, err;
  two_sum(sh, p, s, err);
  sh = s;
  sl += err + e;
}

__device__ __forceinline__ double df_to_double(float h, float l) { return (double)h + (double)l; }

}  // namespace

// hi[i] = fl32(x[i]), lo[i] = fl32(x[i] - hi[i]); flag = 1 if some |x| > 2^100
__global__ void k_split_df64(int64_t count, const double* __restrict__ x, float* __restrict__ hi,
                             float* __restrict__ lo, int* __restrict__ flag) {
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = __double2float_rn(v);
    hi[i] = h;
    lo[i] = __double2float_rn(v - (double)h);
    bad |= (int)(((__double_as_longlong(v) >> 52) & 0x7ff) > kDfBigExp);  // also Inf / NaN
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

int launch_split_df64(pase_ctx* h, int64_t count, const double* x, float* hi, float* lo, int* flag) {
  if (count == 0) return PASE_OK;
  int64_t g = (count + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_split_df64<<<(unsigned)g, 256, 0, h->stream>>>(count, x, hi, lo, flag);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// MODE CSR_MV_AM: Y1 = A X, Y2 = M X.  MODE CSR_EIGRES: Y1 = (M X) diag(lam) - A X (if Y1)
// and per-block column sums of |Y1|^2 and |M X|^2 (FP64) into partial[block][2m].
// tpr = m / 4 threads per row, each owning a float4 column slice of X's hi and lo blocks.
template <int MODE>
__global__ void __launch_bounds__(512) k_csr_df64(int64_t n, int m, int tpr, int rpb, const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col, const float* __restrict__ ah,
                                                  const float* __restrict__ al, const float* __restrict__ mh,
                                                  const float* __restrict__ ml, const float* __restrict__ xh,
                                                  const float* __restrict__ xl, const double* __restrict__ lam,
                                                  double* __restrict__ Y1, double* __restrict__ Y2,
                                                  double* __restrict__ partial) {
  const int tx = threadIdx.x % tpr;
  const int ty = threadIdx.x / tpr;
  const bool active = ty < rpb;
  const int c0 = tx * 4;
  double sr[4] = {0.0, 0.0, 0.0, 0.0}, sm[4] = {0.0, 0.0, 0.0, 0.0};
  float lh[4], ll[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double lv = (MODE == CSR_EIGRES && active) ? lam[c0 + v] : 0.0;
    lh[v] = __double2float_rn(lv);
    ll[v] = __double2float_rn(lv - (double)lh[v]);
  }
  if (active) {
    for (int64_t row = (int64_t)blockIdx.x * rpb + ty; row < n; row += (int64_t)gridDim.x * rpb) {
      float a1h[4] = {0.f, 0.f, 0.f, 0.f}, a1l[4] = {0.f, 0.f, 0.f, 0.f};
      float a2h[4] = {0.f, 0.f, 0.f, 0.f}, a2l[4] = {0.f, 0.f, 0.f, 0.f};
      const int64_t k0 = rowptr[row], k1 = rowptr[row + 1];
      for (int64_t k = k0; k < k1; ++k) {
        const int64_t c = col[k];
        const float vah = ah[k], val = al[k], vmh = mh[k], vml = ml[k];
        const float4 h4 = __ldg(reinterpret_cast<const float4*>(xh + c * m + c0));
        const float4 l4 = __ldg(reinterpret_cast<const float4*>(xl + c * m + c0));
        const float xhv[4] = {h4.x, h4.y, h4.z, h4.w}, xlv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          df_mac(a1h[v], a1l[v], vah, val, xhv[v], xlv[v]);
          df_mac(a2h[v], a2l[v], vmh, vml, xhv[v], xlv[v]);
        }
      }
      const int64_t o = row * m + c0;
      if (MODE == CSR_MV_AM) {
        *reinterpret_cast<double2*>(Y1 + o) = make_double2(df_to_double(a1h[0], a1l[0]), df_to_double(a1h[1], a1l[1]));
        *reinterpret_cast<double2*>(Y1 + o + 2) = make_double2(df_to_double(a1h[2], a1l[2]), df_to_double(a1h[3], a1l[3]));
        *reinterpret_cast<double2*>(Y2 + o) = make_double2(df_to_double(a2h[0], a2l[0]), df_to_double(a2h[1], a2l[1]));
        *reinterpret_cast<double2*>(Y2 + o + 2) = make_double2(df_to_double(a2h[2], a2l[2]), df_to_double(a2h[3], a2l[3]));
      } else {
        double r[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          // (M x) * lambda - A x in double-float, then widened
          float ph, pl;
          {
            const float mh2 = a2h[v] + a2l[v];  // renormalise the M x sum
            const float ml2 = a2l[v] - (mh2 - a2h[v]);
            ph = mh2 * lh[v];
            pl = fmaf(mh2, lh[v], -ph);
            pl = fmaf(mh2, ll[v], fmaf(ml2, lh[v], pl));
            sm[v] = fma(df_to_double(mh2, ml2), df_to_double(mh2, ml2), sm[v]);
          }
          float s, e;
          two_sum(ph, -a1h[v], s, e);
          e += pl - a1l[v];
          r[v] = df_to_double(s, e);
          sr[v] = fma(r[v], r[v], sr[v]);
        }
        if (Y1) {
          *reinterpret_cast<double2*>(Y1 + o) = make_double2(r[0], r[1]);
          *reinterpret_cast<double2*>(Y1 + o + 2) = make_double2(r[2], r[3]);
        }
      }
    }
  }
  if (MODE == CSR_EIGRES) {
    // block reduction of the column sums: red[2][rpb][m] with rpb * m <= 512 * 4
    __shared__ double red[2 * 512 * 4];
    if (active) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        red[ty * m + c0 + v] = sr[v];
        red[rpb * m + ty * m + c0 + v] = sm[v];
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * m; j += blockDim.x) {
      const int half = j / m, c = j % m;
      double s = 0.0;
      for (int r = 0; r < rpb; ++r) s += red[half * rpb * m + r * m + c];
      partial[(int64_t)blockIdx.x * 2 * m + j] = s;
    }
  }
}

int launch_csr_df64(pase_ctx* h, int mode, int m, const DevCSR& A, const float* ah, const float* al,
                    const float* mh, const float* ml, const float* xh, const float* xl, const double* lam,
                    double* Y1, double* Y2, double* partial, int* nblocks_out) {
  if (m % 8 != 0 || m <= 0 || m / 4 > 512) return fail(PASE_ERR_INVALID_ARG, "launch_csr_df64: bad m");
  if (mode != CSR_MV_AM && mode != CSR_EIGRES) return fail(PASE_ERR_INVALID_ARG, "launch_csr_df64: bad mode");
  const int tpr = m / 4;
  int bs = A.block > 0 ? A.block : 256;
  if (bs < tpr) bs = ((tpr + 31) / 32) * 32;
  if (bs > 512) bs = 512;
  const int rpb = bs / tpr;
  int64_t g = (A.nrows + rpb - 1) / rpb;
  if (g < 1) g = 1;
  if (mode == CSR_EIGRES && g > kReduceBlocksHost) g = kReduceBlocksHost;
  const int grid = (int)g;
  if (nblocks_out) *nblocks_out = grid;
  if (A.nrows == 0) return PASE_OK;
  int prof_id = -1;
  if (h->prof_kernel >= 0 && mode == CSR_MV_AM) prof_id = PASE_KERNEL_SPMM_AM_FP64;
  prof_begin(h, prof_id);
  if (mode == CSR_MV_AM)
    k_csr_df64<CSR_MV_AM><<<grid, bs, 0, h->stream>>>(A.nrows, m, tpr, rpb, A.rowptr, A.col, ah, al, mh, ml, xh, xl,
                                                      lam, Y1, Y2, partial);
  else
    k_csr_df64<CSR_EIGRES><<<grid, bs, 0, h->stream>>>(A.nrows, m, tpr, rpb, A.rowptr, A.col, ah, al, mh, ml, xh, xl,
                                                       lam, Y1, Y2, partial);
  prof_end(h, prof_id);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

}  // namespace pase
