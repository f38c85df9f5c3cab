// The two dense FP64 contractions of the path on the BF16 tensor cores, with FP64
// accuracy:
//   * Y = X C for a tall block X [n][k1] and a small C [k1][k2] (k1, k2 <= 128, even):
//     the prolongation W C_W of Alg. 3 step 6.  One launch covers k1, k2 <= 64; wider
//     products run as 64-wide blocks.
//   * the Gram blocks W^T (A_h W), W^T (M_h W) of Alg. 3 step 4 (second part of the file).
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
//     the two lowest diagonals shifted right with rounding) and builds the double
//     T 2^{e_r + f_j - 56} from its bits with integer instructions (FP64 instructions
//     run at ~2 per clock per SM on this part).
// Error: the dropped diagonals d >= 10 (at most ~2^-52 2^{e_r + f_j}), the rounded shifts
// (2^{e_r + f_j - 56}) and the digit rounding (2^{e_r + f_j - 61}): a few units of 2^-53
// relative to max_k |x_rk| max_k |c_kj|, plus the rounding of the result to double;
// on random blocks with K = 56 the entrywise relative error is below the FP64 GEMM's.
// Rows or columns with an Inf or NaN are recomputed in plain FP64 (so they propagate as
// in an FP64 product).
//
// Layout: tiles of 128 rows (M = 128), K and N padded to multiples of 16 with zeros.
// Shared memory holds the 8 A slices [128 x K] and 8 B slices [N x K] in the canonical
// K-major core-matrix layout (8 rows x 16 bytes): 192 KB at K = N = 64, one CTA of 16
// warps per SM, persistent over tiles; the next tile's X rows are loaded into registers
// while the tensor cores work on the current one.
#include <cuda_bf16.h>

#include "pase_internal.h"
#include "tc_util.h"

namespace pase {

constexpr int kSgM = 128;       // rows per tile
constexpr int kSgThreads = 512;  // 16 warps: the slicing and the epilogue are latency-bound
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

// The 36 slice products of one K block into the 8 diagonal accumulators (TMEM columns
// (d - 2) np ...): fully unrolled, descriptors formed by adding compile-time offsets to
// the two base descriptors (the 14-bit address field cannot carry: shared memory is
// below 256 KB).  strideA16 / strideB16: slice strides in 16-byte units.  fresh: the
// first product of each diagonal overwrites the accumulator.
template <int KSTEPS>
__device__ __forceinline__ void sg_issue_products(uint32_t tmem, int np, uint64_t descA0, uint64_t descB0,
                                                  uint32_t strideA16, uint32_t strideB16, uint32_t idesc,
                                                  bool fresh) {
#pragma unroll
  for (int d = 2; d <= kSgDigits + 1; ++d) {
    const uint32_t dcol = tmem + (uint32_t)((d - 2) * np);
#pragma unroll
    for (int p = 1; p <= kSgDigits; ++p) {
      const int q = d - p;
      if (q < 1 || q > kSgDigits) continue;
#pragma unroll
      for (int s = 0; s < KSTEPS; ++s) {
        const bool first = p == (d - kSgDigits > 1 ? d - kSgDigits : 1) && s == 0;
        const uint64_t da = descA0 + (uint64_t)((p - 1) * strideA16 + s * 16);
        const uint64_t db = descB0 + (uint64_t)((q - 1) * strideB16 + s * 16);
        const uint32_t accf = (first && fresh) ? 0u : 1u;
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
                     "l"(da), "l"(db), "r"(idesc), "r"(accf));
      }
    }
  }
}

template <int KP>
__global__ void __launch_bounds__(kSgThreads, 1)
    k_ts_gemm_split(int64_t n, int k1, int k2, int np, const double* __restrict__ X, int64_t ldx,
                    const double* __restrict__ C, int ldc, double* __restrict__ Y, int64_t ldy, int beta,
                    uint32_t tmem_cols, int* __restrict__ err) {
  static_assert(KP % 16 == 0 && KP <= 64, "K tile");
  // threads per row in the load phase: the largest divisor of KP / 8 up to 4
  constexpr int RP = (KP / 8) % 4 == 0 ? 4 : ((KP / 8) % 3 == 0 ? 3 : ((KP / 8) % 2 == 0 ? 2 : 1));
  constexpr int KH = KP / RP;  // K values per loading thread (a multiple of 8)
  static_assert(KH % 8 == 0, "load chunks of 8");
  extern __shared__ __align__(1024) uint8_t sg_smem[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(sg_smem);  // [8][128 x KP]
  __nv_bfloat16* sB = sA + (size_t)kSgDigits * kSgM * KP;          // [8][np x KP]
  __shared__ int sEx[kSgThreads];
  __shared__ int sFx[64];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int strideA = kSgM * KP, strideB = np * KP;

  // A-slice chunks that only hold K padding (k >= k1) stay zero: clear them once
  for (int i = tid; i < kSgDigits * kSgM * KP / 8; i += kSgThreads)
    reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
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

  // load-phase role: row lr of the tile, K part lh (threads with lh >= RP only wait)
  const int lr = tid & (kSgM - 1), lh = tid >> 7;
  const bool loader = lh < RP;
  const int64_t ntiles = (n + kSgM - 1) / kSgM;
  double xv[KH];
  auto load_tile = [&](int64_t tile) {
    const int64_t row = tile * kSgM + lr;
    const bool ok = loader && row < n;
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
    e = sEx[lr];
#pragma unroll
    for (int q = 1; q < RP; ++q) e = max(e, sEx[lr + q * kSgM]);
#pragma unroll
    for (int c8 = 0; c8 < (loader ? KH / 8 : 0); ++c8) {
      const int kc = lh * (KH / 8) + c8;
      if (kc * 8 >= k1) continue;  // padding only: still zero
      uint64_t z[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) z[c] = sg_fixed(xv[c8 * 8 + c], e);
      sg_store_chunk(z, sA + (lr >> 3) * (KP * 8) + kc * 64 + (lr & 7) * 8, strideA);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // ---- 36 slice products per K step into the 8 diagonal accumulators
    if (tid == 0) {
      sg_issue_products<KP / 16>(tmem, np, umma_desc(aBase, 128, KP * 16), umma_desc(bBase, 128, KP * 16),
                                 (uint32_t)(strideA / 8), (uint32_t)(strideB / 8), idesc, true);
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
    // ---- epilogue: warp -> 32 TMEM lanes (rows) x a quarter of the columns
    const int lq = warp & 3, part = warp >> 2, npart = np / 4;  // npart: a multiple of 4
    const int er = lq * 32 + lane;
    const int64_t row = tile * kSgM + er;
    int erx = sEx[er];
#pragma unroll
    for (int q = 1; q < RP; ++q) erx = max(erx, sEx[er + q * kSgM]);
    const uint32_t lane_addr = tmem + ((uint32_t)(lq * 32) << 16);
    for (int c0 = part * npart; c0 < (part + 1) * npart; c0 += 4) {
      uint32_t v[8][4];
#pragma unroll
      for (int d = 0; d < 8; ++d)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3])
                     : "r"(lane_addr + (uint32_t)(d * np + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < n) {
        double out[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          int64_t T = 0;
#pragma unroll
          for (int d = 0; d < 6; ++d) T += (int64_t)__float2int_rn(__uint_as_float(v[d][c])) * (1ll << (44 - 8 * d));
          T += (int64_t)((__float2int_rn(__uint_as_float(v[6][c])) + (1 << 3)) >> 4);  // to nearest
          T += (int64_t)((__float2int_rn(__uint_as_float(v[7][c])) + (1 << 11)) >> 12);
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
          for (int c = 0; c < 4; ++c)
            if (c0 + c < k2) out[c] += yr[c];
        }
        if (c0 + 4 <= k2) {
          *reinterpret_cast<double2*>(yr) = make_double2(out[0], out[1]);
          *reinterpret_cast<double2*>(yr + 2) = make_double2(out[2], out[3]);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c)
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

// ------------------------------------------------------------------ Gram blocks
// D = A^T B over the rows of a tall block pair (Alg. 3 step 4: W^T (A_h W), W^T (M_h W)),
// with A = [A0 | A1] (two blocks of at most 64 columns, M = 128) and B at most 64
// columns, by the same digit splitting with the scales taken per column over all rows
// (a pre-pass, k_colexp).  Each CTA takes a contiguous row range in chunks of 64 rows (the
// MMA K); the 8 diagonal accumulators collect two chunks (128 rows: |D_d| <= 128 x 114688
// < 2^24, still exact) and are then drained into per-thread 64-bit integer sums
// T += sum_d D_d 2^{52 - 8d} (unit 2^{e_i + f_j - 48}; the three lowest diagonals shifted
// right with rounding, so the per-drain error is unbiased), which stay below 2^63 for up
// to 2^14 rows per CTA.  The CTA writes its sums as doubles to partial[cta][128][np]; a
// reduction kernel adds the CTAs in FP64.  On random blocks the error relative to
// sum_r |a_ri||b_rj| is below that of the FP64 Gram kernel.
constexpr int kGsK = 64;          // rows per chunk (MMA K)
constexpr int kGsDrainChunks = 2;  // chunks per accumulation
constexpr int64_t kGsMaxRowsPerCta = 1 << 14;
constexpr int kGsU0 = 48;          // T unit 2^{e_i + f_j - 48}
constexpr int kGsThreads = 512;     // 16 warps: the slicing is latency-bound
constexpr int kGsWarpParts = kGsThreads / 128;  // warps sharing one TMEM lane quarter
constexpr int kGsOut = 64 / kGsWarpParts;       // accumulator columns per thread (np <= 64)
constexpr int kGsItems = (kSgM * 8 + 64 * 8) / kGsThreads;  // slicing items per thread

// column exponents (sg_bexp + 2048, so 0 = "no value yet") by atomicMax; blockIdx.y
// selects one of three [n][ld] arrays, columns [c0, c0 + m), m <= 64
struct ColexpArgs {
  const double* x[3];
  int* out[3];
};
__global__ void __launch_bounds__(256) k_colexp(int64_t n, int m, int64_t ld, ColexpArgs a) {
  __shared__ int se[256];
  const int y = blockIdx.y;
  const double* __restrict__ X = y == 0 ? a.x[0] : (y == 1 ? a.x[1] : a.x[2]);
  int* out = y == 0 ? a.out[0] : (y == 1 ? a.out[1] : a.out[2]);
  const int c = threadIdx.x & 63, r4 = threadIdx.x >> 6;
  int e = 0;
  if (c < m) {
    const int64_t step = (int64_t)gridDim.x * 16;
    for (int64_t rb = (int64_t)blockIdx.x * 16 + r4; rb < n; rb += step) {
      double v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t r = rb + 4 * k;
        v[k] = r < n ? X[r * ld + c] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (rb + 4 * k < n) e = max(e, sg_bexp(v[k]) + 2048);
    }
  }
  se[threadIdx.x] = e;
  __syncthreads();
  if (threadIdx.x < 64 && c < m) {
    const int v = max(max(se[c], se[c + 64]), max(se[c + 128], se[c + 192]));
    if (v > 0) atomicMax(out + c, v);
  }
}

__global__ void __launch_bounds__(kGsThreads, 1)
    k_gram_split(int64_t n, int64_t rows_per_cta, const double* __restrict__ A0, int64_t lda0, int na0,
                 const double* __restrict__ A1, int64_t lda1, int na1, const double* __restrict__ B, int64_t ldb,
                 int nbc, int np, const int* __restrict__ aexp0, const int* __restrict__ aexp1,
                 const int* __restrict__ bexp, double* __restrict__ partial, uint32_t tmem_cols,
                 int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t sg_smem[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(sg_smem);  // [8][128 x 64]
  __nv_bfloat16* sB = sA + (size_t)kSgDigits * kSgM * kGsK;        // [8][np x 64]
  __shared__ int sAe[kSgM], sBe[64];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int strideA = kSgM * kGsK, strideB = np * kGsK;
  if (tid < kSgM) {
    int e = 0;
    if (tid < 64 && tid < na0) e = aexp0[tid];
    if (tid >= 64 && tid - 64 < na1) e = aexp1[tid - 64];
    sAe[tid] = e - 2048;
  }
  if (tid < 64) sBe[tid] = (tid < nbc ? bexp[tid] : 0) - 2048;
  // slices of padding columns (beyond na0, na1, nbc) stay zero: clear both buffers once
  for (int i = tid; i < (kSgDigits * kSgM * kGsK + kSgDigits * np * kGsK) / 8; i += kGsThreads)
    reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
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
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(n, r0 + rows_per_cta);
  // drain role: TMEM lane (A column) er, B columns [jb, jb + np/2)
  const int npart = np / kGsWarpParts;  // columns per warp (a multiple of 4)
  const int lq = warp & 3, er = lq * 32 + lane, jb = (warp >> 2) * npart;
  const uint32_t lane_addr = tmem + ((uint32_t)(lq * 32) << 16);
  int64_t acc[kGsOut];
#pragma unroll
  for (int c = 0; c < kGsOut; ++c) acc[c] = 0;
  uint32_t phase = 0;
  bool ok = true;
  int chunk = 0;
  // one slicing item = 8 consecutive rows of one column (A: 128 x 8 items, B: np x 8);
  // lanes take consecutive columns, so each load instruction reads contiguous row segments
  const int nitems = kSgM * 8 + np * 8;
  auto item = [&](int it, const double*& src, int64_t& ld, int& col, bool& valid, int& e, int& kg,
                  __nv_bfloat16*& dst, int& stride) {
    if (it < kSgM * 8) {
      const int i = it % kSgM;
      kg = it / kSgM;
      const bool hi = i >= 64;
      col = hi ? i - 64 : i;
      src = hi ? A1 : A0;
      ld = hi ? lda1 : lda0;
      valid = col < (hi ? na1 : na0);
      e = sAe[i];
      dst = sA + (i >> 3) * (kGsK * 8) + kg * 64 + (i & 7) * 8;
      stride = strideA;
    } else {
      const int j = (it - kSgM * 8) % np;
      kg = (it - kSgM * 8) / np;
      col = j;
      src = B;
      ld = ldb;
      valid = j < nbc;
      e = sBe[j < 64 ? j : 0];
      dst = sB + (j >> 3) * (kGsK * 8) + kg * 64 + (j & 7) * 8;
      stride = strideB;
    }
  };
  double pv[kGsItems][8];  // raw values of this thread's items of the next chunk
  auto load_chunk = [&](int64_t rb) {
#pragma unroll
    for (int q = 0; q < kGsItems; ++q) {
      const int it = tid + q * kGsThreads;
      const double* src = nullptr;
      int64_t ld = 0;
      int col = 0, e = 0, kg = 0, stride = 0;
      bool valid = false;
      __nv_bfloat16* dst = nullptr;
      if (it < nitems) item(it, src, ld, col, valid, e, kg, dst, stride);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t r = rb + kg * 8 + c;
        pv[q][c] = (valid && r < r1) ? __ldg(src + r * ld + col) : 0.0;
      }
    }
  };
  if (r0 < r1) load_chunk(r0);
  for (int64_t rb = r0; rb < r1; rb += kGsK, ++chunk) {
    // ---- digit slices of rows [rb, rb + 64) from the prefetched values
#pragma unroll
    for (int q = 0; q < kGsItems; ++q) {
      const int it = tid + q * kGsThreads;
      if (it < nitems) {
        const double* src;
        int64_t ld;
        int col, e, kg, stride;
        bool valid;
        __nv_bfloat16* dst;
        item(it, src, ld, col, valid, e, kg, dst, stride);
        if (!valid) continue;  // padding column: its slices stay zero
        uint64_t z[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) z[c] = sg_fixed(pv[q][c], e);
        sg_store_chunk(z, dst, stride);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      sg_issue_products<kGsK / 16>(tmem, np, umma_desc(aBase, 128, kGsK * 16), umma_desc(bBase, 128, kGsK * 16),
                                   (uint32_t)(strideA / 8), (uint32_t)(strideB / 8), idesc,
                                   (chunk % kGsDrainChunks) == 0);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    if (rb + kGsK < r1) load_chunk(rb + kGsK);  // next chunk's rows while the tensor cores run
    const uint32_t done = mbar_wait_bounded(smem_u32(&mbar), phase, 1 << 22);
    if (!__syncthreads_and((int)done)) {  // (uniform) give up: report, let the MMAs finish, stop
      if (tid == 0) atomicExch(err, 1);
      mbar_wait_bounded(smem_u32(&mbar), phase, 1 << 22);
      ok = false;
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // ---- drain after every second chunk and after the last
    if ((chunk % kGsDrainChunks) == kGsDrainChunks - 1 || rb + kGsK >= r1) {
#pragma unroll
      for (int cb = 0; cb < kGsOut / 4; ++cb) {
        if (cb * 4 < npart) {  // warp-uniform
          uint32_t v[8][4];
#pragma unroll
          for (int d = 0; d < 8; ++d)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3])
                         : "r"(lane_addr + (uint32_t)(d * np + jb + cb * 4)));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            int64_t T = 0;
#pragma unroll
            for (int d = 0; d < 5; ++d)  // diagonals 2..6: shifts 36, 28, 20, 12, 4
              T += (int64_t)__float2int_rn(__uint_as_float(v[d][c])) * (1ll << (36 - 8 * d));
            T += (int64_t)((__float2int_rn(__uint_as_float(v[5][c])) + (1 << 3)) >> 4);  // to nearest
            T += (int64_t)((__float2int_rn(__uint_as_float(v[6][c])) + (1 << 11)) >> 12);
            T += (int64_t)((__float2int_rn(__uint_as_float(v[7][c])) + (1 << 19)) >> 20);
            acc[cb * 4 + c] += T;
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // slices and (after a drain) the accumulators are reused
  }
  if (ok) {
    // ---- the CTA's sums as doubles; Inf/NaN columns summed directly in FP64
    double* out = partial + ((int64_t)blockIdx.x * kSgM + er) * np;
    const int ie = sAe[er];
    const bool hi = er >= 64;
    const int icol = hi ? er - 64 : er;
    const bool ivalid = icol < (hi ? na1 : na0);
#pragma unroll
    for (int c = 0; c < kGsOut; ++c) {
      const int j = jb + c;
      if (c < npart) {
        double vout = 0.0;
        if (ivalid && j < nbc) {
          const int je = sBe[j];
          if (ie == 2047 || je == 2047) {
            const double* a = hi ? A1 : A0;
            const int64_t la = hi ? lda1 : lda0;
            double s2 = 0.0;
            for (int64_t r = r0; r < r1; ++r) s2 = fma(a[r * la + icol], B[r * ldb + j], s2);
            vout = s2;
          } else {
            vout = sg_to_double(acc[c], ie + je - 2044 - kGsU0);
          }
        }
        out[j] = vout;
      }
    }
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// G_g[p][q] = G_g[q][p] = sum_b partial[b][i][j] for the entries of this launch with
// p = n0 + j <= q = column of A index i (the upper triangle of W^T Y, mirrored, as in the
// FP64 path); A index i < 64 belongs to G0 (column c0 + i), i >= 64 to G1 (c1 + i - 64).
__global__ void k_gram_split_reduce(int nb, int np, const double* __restrict__ partial, int na0, int na1, int nbc,
                                    double* __restrict__ G0, int c0, double* __restrict__ G1, int c1, int n0,
                                    int ldg) {
  const int total = kSgM * np;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int i = idx / np, j = idx % np;
    const bool hi = i >= 64;
    const int ic = hi ? i - 64 : i;
    if (ic >= (hi ? na1 : na0) || j >= nbc) continue;
    const int q = (hi ? c1 : c0) + ic, p = n0 + j;
    if (p > q) continue;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[((int64_t)b * kSgM + i) * np + j];
    double* G = hi ? G1 : G0;
    G[(int64_t)p * ldg + q] = s;
    G[(int64_t)q * ldg + p] = s;
  }
}

// CTAs of the split Gram over n rows: at least one per SM, at most 2^14 rows each, whole
// 64-row chunks; *rows_per_cta receives the rows of each.
static int64_t gram_split_grid(int64_t n, int num_sms, int64_t* rows_per_cta) {
  int64_t grid = std::max<int64_t>(num_sms, (n + kGsMaxRowsPerCta - 1) / kGsMaxRowsPerCta);
  grid = std::max<int64_t>(1, std::min<int64_t>(grid, (n + kGsK - 1) / kGsK));
  int64_t rpc = (n + grid - 1) / grid;
  rpc = (rpc + kGsK - 1) / kGsK * kGsK;
  if (rows_per_cta) *rows_per_cta = rpc;
  return (n + rpc - 1) / rpc;
}

bool ts_gram2_split_ok(int64_t n, int m, int num_sms, const Work& w) {
  if (m < 2 || m > 128 || (m % 2) != 0) return false;
  const int64_t np = m <= 64 ? (m + 15) / 16 * 16 : 64;  // widest B block of a launch
  const int64_t need = std::max<int64_t>(1, gram_split_grid(n, num_sms, nullptr)) * kSgM * np;
  return (int64_t)(w.partial_bytes / sizeof(double)) >= need;  // every CTA's partials fit
}

// GA = W^T Y1 and GB = W^T Y2 (symmetric, upper triangle mirrored), all [n][m], m <= 128
// even; colexp: device scratch of 3 x 128 ints.
int ts_gram2_split(pase_ctx* h, int64_t n, int m, const double* W, const double* Y1, const double* Y2, double* GA,
                   double* GB, int ldg, int* colexp, int* err) {
  if (n == 0 || m == 0) return PASE_OK;
  Work& w = h->w;
  // column exponents of Y1, Y2, W
  PASE_CUDA(cudaMemsetAsync(colexp, 0, 3 * 128 * sizeof(int), h->stream));
  const int ceg = (int)std::min<int64_t>((n + 15) / 16, (int64_t)h->num_sms * 4);
  for (int c0 = 0; c0 < m; c0 += 64) {
    ColexpArgs a{{Y1 + c0, Y2 + c0, W + c0}, {colexp + c0, colexp + 128 + c0, colexp + 256 + c0}};
    k_colexp<<<dim3((unsigned)ceg, 3), 256, 0, h->stream>>>(n, std::min(64, m - c0), m, a);
    h->launches++;
  }
  PASE_CUDA(cudaGetLastError());
  int64_t rpc = 0;
  const int64_t grid = gram_split_grid(n, h->num_sms, &rpc);
  const size_t smem = std::max<size_t>(sg_smem_bytes(kGsK, 64), 116 * 1024);
  PASE_TRY(ensure_max_smem((const void*)k_gram_split, 200 * 1024));
  auto launch = [&](const double* A0, int na0, const int* e0, const double* A1, int na1, const int* e1,
                    const double* Bp, int nbc, const int* eb, double* G0, int cc0, double* G1, int cc1,
                    int n0) -> int {
    const int np = (nbc + 15) / 16 * 16;
    if ((int64_t)grid * kSgM * np > (int64_t)(w.partial_bytes / sizeof(double)))
      return fail(PASE_ERR_INVALID_ARG, "ts_gram2_split: partial buffer too small");
    uint32_t cols = 32;
    while (cols < (uint32_t)(8 * np)) cols <<= 1;
    k_gram_split<<<(unsigned)grid, kGsThreads, smem, h->stream>>>(n, rpc, A0, m, na0, A1, m, na1, Bp, m, nbc, np,
                                                                  e0, e1, eb, w.partial, cols, err);
    h->launches++;
    PASE_CUDA(cudaGetLastError());
    const int total = kSgM * np;
    k_gram_split_reduce<<<(total + 255) / 256, 256, 0, h->stream>>>((int)grid, np, w.partial, na0, na1, nbc, G0,
                                                                     cc0, G1, cc1, n0, ldg);
    h->launches++;
    PASE_CUDA(cudaGetLastError());
    return PASE_OK;
  };
  int* eY1 = colexp;
  int* eY2 = colexp + 128;
  int* eW = colexp + 256;
  if (m <= 64) return launch(Y1, m, eY1, Y2, m, eY2, W, m, eW, GA, 0, GB, 0, 0);
  // wider: per Gram, A = [Y[:, 0:64] | Y[:, 64:m]], B = W in two column blocks
  const int b0 = ((m / 2) + 1) & ~1;
  const int nbs[2] = {b0, m - b0};
  for (int g = 0; g < 2; ++g) {
    const double* Y = g == 0 ? Y1 : Y2;
    const int* eY = g == 0 ? eY1 : eY2;
    double* G = g == 0 ? GA : GB;
    int n0 = 0;
    for (int k = 0; k < 2; n0 += nbs[k], ++k)
      PASE_TRY(launch(Y, 64, eY, Y + 64, m - 64, eY + 64, W + n0, nbs[k], eW + n0, G, 0, G, 64, n0));
  }
  return PASE_OK;
}

}  // namespace pase
