// Y = X C for a tall block X [n][k1] and a small C [k1][k2] (k1, k2 <= 128, even) on the
// BF16 tensor cores with FP64 accuracy: the prolongation W C_W of Alg. 3 step 6.  One
// launch covers k1, k2 <= 64; wider products run as 64-wide blocks.
//
// Error-free splitting (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication", Numer.
// Algorithms 59, 2012), in the integer-digit form used here:
//   * every row r of X gets a power-of-two scale 2^{e_r} within a factor 2 above its
//     largest entry (subnormals included), and every entry becomes the 64-bit integer
//     Y = round(x 2^{62 - e_r}), |Y| < 2^62;
//   * Y is written in 8 balanced base-256 digits a_1..a_8 in [-128, 127] (the bytes of
//     Y + 0x8080808080808080, less 128), so x = 2^{e_r + 2} sum_p a_p 2^{-8p} up to
//     2^{e_r - 63}; the columns of C the same way (b_1..b_8, scale 2^{f_j + 2});
//   * the digits are exact in bfloat16, a digit product is at most 2^14, and the
//     tensor core sums the products of one anti-diagonal d = p + q (at most 8 slice
//     pairs times K <= 64 terms, |sum| < 2^23) exactly in its FP32 accumulator:
//     D_d = sum_{p+q=d} A_p B_q, one TMEM accumulator per d = 2..9 (36 MMAs per K step);
//   * the epilogue recombines T = sum_d D_d 2^{60 - 8d} in 64-bit integers (|T| < 2^62;
//     the two lowest diagonals shifted right, floor) and builds the double
//     T 2^{e_r + f_j - 56} from its bits with integer instructions (FP64 instructions
//     run at ~2 per clock per SM on this part).
// Error: the dropped diagonals d >= 10 (at most ~2^-52 2^{e_r + f_j}), the floor shifts
// (2^{e_r + f_j - 55}) and the digit rounding (2^{e_r + f_j - 61}): a few units of 2^-53
// relative to max_k |x_rk| max_k |c_kj|, plus the rounding of the result to double;
// on random blocks with K = 56 the entrywise relative error is below the FP64 GEMM's.
// Rows or columns with an Inf or NaN are recomputed in plain FP64 (so they propagate as
// in an FP64 product).
//
// Layout: tiles of 128 rows (M = 128), K and N padded to multiples of 16 with zeros.
// Shared memory holds the 8 A slices [128 x K] and 8 B slices [N x K] in the canonical
// K-major core-matrix layout (8 rows x 16 bytes): 192 KB at K = N = 64, one CTA per SM,
// persistent over tiles; the next tile's X rows are loaded into registers while the
// tensor cores work on the current one.
#include <cuda_bf16.h>

#include "pase_internal.h"
#include "tc_util.h"

namespace pase {

constexpr int kSgM = 128;       // rows per tile
constexpr int kSgThreads = 256;
constexpr int kSgDigits = 8;

__host__ __device__ inline size_t sg_smem_bytes(int kp, int np) {
  return (size_t)kSgDigits * kSgM * kp * 2 + (size_t)kSgDigits * np * kp * 2;
}

// exponent used for scaling: the biased exponent E of a normal value (2047 = Inf/NaN);
// for a subnormal the same quantity from its leading bit (<= 0), so that 2^{E - 1022}
// stays within a factor 2 of |x|; kSgZeroExp for zero (never the maximum of a nonzero row)
constexpr int kSgZeroExp = -1100;
__device__ __forceinline__ int sg_bexp(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E != 0) return E;
  const uint64_t M = b & 0xFFFFFFFFFFFFFull;
  return M == 0 ? kSgZeroExp : (63 - __clzll((long long)M)) - 51;
}

// Y + 0x8080808080808080 with Y = round(x 2^{62 - e}), e = emax - 1022 (emax >= sg_bexp
// of the operand): its bytes are the balanced digits plus 128.  |x| = M 2^{E' - 1075}
// with E' = max(E, 1); for x != 0 the shift E' - emax + 9 is at most 9 (normal) or
// 61 - (leading bit of M) (subnormal), so |Y| < 2^62.
__device__ __forceinline__ uint64_t sg_fixed(double x, int emax) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  uint64_t M = b & 0xFFFFFFFFFFFFFull;
  if (E != 0) M |= 1ull << 52;
  const int s = (E == 0 ? 1 : E) - emax + 9;
  uint64_t Y;
  if (M == 0) Y = 0;
  else if (s >= 0) Y = M << s;
  else if (s > -63) Y = (M + (1ull << (-s - 1))) >> (-s);  // to nearest, ties away from zero
  else Y = 0;
  if (b >> 63) Y = 0ull - Y;
  return Y + 0x8080808080808080ull;
}

// digit byte `sel` (0..3) of a 32-bit word -> the bfloat16 bit pattern of (byte - 128),
// in the upper half of the returned word (exact: |digit| <= 128 has <= 8 significant bits)
__device__ __forceinline__ uint32_t sg_digit_f32(uint32_t word, uint32_t sel) {
  const uint32_t f = __byte_perm(word, 0x4B000000u, 0x7540u | sel);  // float 2^23 + byte
  return __float_as_uint(__uint_as_float(f) - 8388736.0f);         // - (2^23 + 128)
}

// Write the 8 digit slices of 8 consecutive values (one 16-byte chunk per slice).
// z[c] = sg_fixed of value c; slice p (0 = most significant digit) at base + p * stride.
__device__ __forceinline__ void sg_store_chunk(const uint64_t (&z)[8], __nv_bfloat16* base, int stride) {
#pragma unroll
  for (int p = 0; p < kSgDigits; ++p) {
    const int byte = 7 - p;  // most significant byte first
    const int half = byte >> 2;
    const uint32_t sel = (uint32_t)(byte & 3);
    uint32_t w[4];
#pragma unroll
    for (int c = 0; c < 8; c += 2) {
      const uint32_t lo = sg_digit_f32(half ? (uint32_t)(z[c] >> 32) : (uint32_t)z[c], sel);
      const uint32_t hi = sg_digit_f32(half ? (uint32_t)(z[c + 1] >> 32) : (uint32_t)z[c + 1], sel);
      w[c >> 1] = __byte_perm(lo, hi, 0x7632u);  // two bfloat16 (upper halves)
    }
    *reinterpret_cast<uint4*>(base + (size_t)p * stride) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// double nearest to T 2^X (integer instructions; ldexp where the result is not normal)
__device__ __forceinline__ double sg_to_double(int64_t T, int X) {
  if (T == 0) return 0.0;
  const uint64_t sgn = (uint64_t)T & 0x8000000000000000ull;
  uint64_t u = T < 0 ? 0ull - (uint64_t)T : (uint64_t)T;
  const int lz = __clzll((long long)u);
  u <<= lz;  // leading bit at 63
  uint64_t mant = u >> 11;
  const uint64_t rest = u & 0x7FFull;
  if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ++mant;  // to nearest even
  int be = X - lz + 63 + 1023;
  if (mant >> 53) {
    mant >>= 1;
    ++be;
  }
  if (be >= 1 && be <= 2046)
    return __longlong_as_double((long long)(sgn | ((uint64_t)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
  return ldexp((double)T, X);
}

template <int KP>
__global__ void __launch_bounds__(kSgThreads, 1)
    k_ts_gemm_split(int64_t n, int k1, int k2, int np, const double* __restrict__ X, int64_t ldx,
                    const double* __restrict__ C, int ldc, double* __restrict__ Y, int64_t ldy, int beta,
                    uint32_t tmem_cols, int* __restrict__ err) {
  static_assert(KP % 16 == 0 && KP <= 64, "K tile");
  constexpr int KH = KP / 2;  // K values per thread in the load phase
  extern __shared__ __align__(1024) uint8_t sg_smem[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(sg_smem);  // [8][128 x KP]
  __nv_bfloat16* sB = sA + (size_t)kSgDigits * kSgM * KP;          // [8][np x KP]
  __shared__ int sEx[kSgThreads];
  __shared__ int sFx[64];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int strideA = kSgM * KP, strideB = np * KP;

  // ---- B slices from C (every CTA; C is at most 64 x 64)
  if (tid < 64) {
    int f = kSgZeroExp;
    if (tid < k2)
      for (int k = 0; k < k1; ++k) f = max(f, sg_bexp(C[(int64_t)k * ldc + tid]));
    sFx[tid] = f;
  }
  __syncthreads();
  for (int ch = tid; ch < np * (KP / 8); ch += kSgThreads) {
    const int j = ch / (KP / 8), kc = ch % (KP / 8);
    uint64_t z[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k = kc * 8 + c;
      const double v = (j < k2 && k < k1) ? C[(int64_t)k * ldc + j] : 0.0;
      z[c] = sg_fixed(v, sFx[j < 64 ? j : 0]);
    }
    sg_store_chunk(z, sB + (j >> 3) * (KP * 8) + kc * 64 + (j & 7) * 8, strideB);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = umma_idesc_bf16(kSgM, np);
  const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB);

  // load-phase role: row lr of the tile, K half lh
  const int lr = tid & (kSgM - 1), lh = tid >> 7;
  const int64_t ntiles = (n + kSgM - 1) / kSgM;
  double xv[KH];
  auto load_tile = [&](int64_t tile) {
    const int64_t row = tile * kSgM + lr;
    const bool ok = row < n;
    const double* src = X + (ok ? row : 0) * ldx + lh * KH;
#pragma unroll
    for (int c = 0; c < KH; c += 2) {
      const int k = lh * KH + c;
      double2 v = make_double2(0.0, 0.0);
      if (ok && k < k1) v = __ldg(reinterpret_cast<const double2*>(src + c));  // k1 even
      xv[c] = v.x;
      xv[c + 1] = v.y;
    }
  };
  if ((int64_t)blockIdx.x < ntiles) load_tile(blockIdx.x);
  uint32_t phase = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- row scale, then the A slices
    int e = kSgZeroExp;
#pragma unroll
    for (int c = 0; c < KH; ++c) e = max(e, sg_bexp(xv[c]));
    sEx[tid] = e;
    __syncthreads();
    e = max(sEx[lr], sEx[lr + kSgM]);
#pragma unroll
    for (int c8 = 0; c8 < KH / 8; ++c8) {
      uint64_t z[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) z[c] = sg_fixed(xv[c8 * 8 + c], e);
      const int kc = lh * (KH / 8) + c8;
      sg_store_chunk(z, sA + (lr >> 3) * (KP * 8) + kc * 64 + (lr & 7) * 8, strideA);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // ---- 36 slice products per K step into the 8 diagonal accumulators
    if (tid == 0) {
#pragma unroll 1
      for (int d = 2; d <= 2 * kSgDigits; ++d) {
        if (d > kSgDigits + 1) break;
        const uint32_t dcol = tmem + (uint32_t)((d - 2) * np);
        bool first = true;
        for (int p = 1; p < d; ++p) {
          const int q = d - p;
          if (p > kSgDigits || q > kSgDigits) continue;
#pragma unroll
          for (int s = 0; s < KP / 16; ++s) {
            const uint64_t da = umma_desc(aBase + (uint32_t)(((p - 1) * strideA + s * 128) * 2), 128, KP * 16);
            const uint64_t db = umma_desc(bBase + (uint32_t)(((q - 1) * strideB + s * 128) * 2), 128, KP * 16);
            const uint32_t acc = first ? 0u : 1u;
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
                         "l"(da), "l"(db), "r"(idesc), "r"(acc));
            first = false;
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    // next tile's rows while the tensor cores run
    if (tile + gridDim.x < ntiles) load_tile(tile + gridDim.x);
    const uint32_t done = mbar_wait_bounded(smem_u32(&mbar), phase, 1 << 22);
    if (!__syncthreads_and((int)done)) {  // (uniform) give up: report, let the MMAs finish, stop
      if (tid == 0) atomicExch(err, 1);
      mbar_wait_bounded(smem_u32(&mbar), phase, 1 << 22);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // ---- epilogue: warp -> 32 TMEM lanes (rows) x half of the columns
    const int lq = warp & 3, chh = warp >> 2;
    const int er = lq * 32 + lane;
    const int64_t row = tile * kSgM + er;
    const int erx = max(sEx[er], sEx[er + kSgM]);
    const uint32_t lane_addr = tmem + ((uint32_t)(lq * 32) << 16);
    for (int c0 = chh * (np / 2); c0 < (chh + 1) * (np / 2); c0 += 8) {
      uint32_t v[8][8];
#pragma unroll
      for (int d = 0; d < 8; ++d)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3]), "=r"(v[d][4]), "=r"(v[d][5]),
                       "=r"(v[d][6]), "=r"(v[d][7])
                     : "r"(lane_addr + (uint32_t)(d * np + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < n) {
        double out[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          int64_t T = 0;
#pragma unroll
          for (int d = 0; d < 6; ++d) T += (int64_t)__float2int_rn(__uint_as_float(v[d][c])) * (1ll << (44 - 8 * d));
          T += (int64_t)(__float2int_rn(__uint_as_float(v[6][c])) >> 4);
          T += (int64_t)(__float2int_rn(__uint_as_float(v[7][c])) >> 12);
          const int j = c0 + c;
          const int fj = sFx[j];
          if (erx == 2047 || fj == 2047) {  // Inf/NaN in the row or the column: plain FP64
            double s = 0.0;
            if (j < k2)
              for (int k = 0; k < k1; ++k) s = fma(X[row * ldx + k], C[(int64_t)k * ldc + j], s);
            out[c] = s;
          } else {
            out[c] = sg_to_double(T, erx + fj - 2100);
          }
        }
        double* yr = Y + row * ldy + c0;
        if (beta) {  // Y += X C (a second K block of a wider product)
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (c0 + c < k2) out[c] += yr[c];
        }
        if (c0 + 8 <= k2) {
#pragma unroll
          for (int c = 0; c < 8; c += 2) *reinterpret_cast<double2*>(yr + c) = make_double2(out[c], out[c + 1]);
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (c0 + c < k2) yr[c] = out[c];
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // A slices, sEx and the accumulators are reused by the next tile
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

bool ts_gemm_split_ok(int k1, int k2, const void* X, int64_t ldx, const void* Y, int64_t ldy) {
  return k1 >= 2 && k1 <= 128 && k2 >= 1 && k2 <= 128 && (k1 % 2) == 0 && (k2 % 2) == 0 && (ldx % 2) == 0 &&
         (ldy % 2) == 0 && ((uintptr_t)X % 16) == 0 && ((uintptr_t)Y % 16) == 0;
}

// one launch: k1, k2 <= 64
static int split_launch(pase_ctx* h, int64_t n, int k1, int k2, const double* X, int64_t ldx, const double* C,
                        int ldc, double* Y, int64_t ldy, int beta, int* err) {
  const int kp = (k1 + 15) / 16 * 16, np = (k2 + 15) / 16 * 16;
  uint32_t cols = 32;
  while (cols < (uint32_t)(8 * np)) cols <<= 1;
  // at least 116 KB so that one CTA (holding up to all 512 TMEM columns) runs per SM
  size_t smem = sg_smem_bytes(kp, np);
  if (smem < 116 * 1024) smem = 116 * 1024;
  const int64_t ntiles = (n + kSgM - 1) / kSgM;
  const int grid = (int)std::min<int64_t>(ntiles, h->num_sms);
  const void* fn;
  switch (kp) {
    case 16: fn = (const void*)k_ts_gemm_split<16>; break;
    case 32: fn = (const void*)k_ts_gemm_split<32>; break;
    case 48: fn = (const void*)k_ts_gemm_split<48>; break;
    default: fn = (const void*)k_ts_gemm_split<64>; break;
  }
  PASE_TRY(ensure_max_smem(fn, 200 * 1024));  // the largest request of any shape (192 KB)
#define PASE_SG_LAUNCH(KP)                                                                                      \
  k_ts_gemm_split<KP><<<grid, kSgThreads, smem, h->stream>>>(n, k1, k2, np, X, ldx, C, ldc, Y, ldy, beta, cols, \
                                                              err)
  switch (kp) {
    case 16: PASE_SG_LAUNCH(16); break;
    case 32: PASE_SG_LAUNCH(32); break;
    case 48: PASE_SG_LAUNCH(48); break;
    default: PASE_SG_LAUNCH(64); break;
  }
#undef PASE_SG_LAUNCH
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// Widths above 64 in blocks of at most 64 (even sizes): Y[:, nb] = sum over K blocks kb of
// X[:, kb] C[kb, nb], the K blocks after the first added to Y in FP64 (one more rounding).
int ts_gemm_split(pase_ctx* h, int64_t n, int k1, int k2, const double* X, int64_t ldx, const double* C, int ldc,
                  double* Y, int64_t ldy, int* err) {
  if (n == 0 || k2 == 0) return PASE_OK;
  if (!ts_gemm_split_ok(k1, k2, X, ldx, Y, ldy)) return fail(PASE_ERR_INVALID_ARG, "ts_gemm_split: unsupported shape");
  auto blocks = [](int k) {  // 1 or 2 blocks of even size <= 64
    if (k <= 64) return std::make_pair(k, 0);
    const int a = ((k / 2) + 1) & ~1;
    return std::make_pair(a, k - a);
  };
  const auto kb = blocks(k1), nb = blocks(k2);
  const int ks[2] = {kb.first, kb.second}, ns[2] = {nb.first, nb.second};
  int n0 = 0;
  for (int j = 0; j < 2 && ns[j] > 0; n0 += ns[j], ++j) {
    int k0 = 0;
    for (int i = 0; i < 2 && ks[i] > 0; k0 += ks[i], ++i)
      PASE_TRY(split_launch(h, n, ks[i], ns[j], X + k0, ldx, C + (int64_t)k0 * ldc + n0, ldc, Y + n0, ldy,
                            i > 0 ? 1 : 0, err));
  }
  return PASE_OK;
}

}  // namespace pase
