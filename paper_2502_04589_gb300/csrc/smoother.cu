// Learned fine-level smoother: a 3^d convolutional network (2 -> 16 -> 16 -> 16 -> 1
// channels, ReLU after the first three layers, zero padding) that replaces the damped
// Jacobi sweeps of the V-cycle on the fine level, x <- x + S(b - A x).  The paper has no
// learned smoother; this is a growth item of the GPU path, defined as follows.
//
// Grid: the fine level is the (n-1)^d interior-node grid of the uniform n^d Q1 mesh,
// node i = sum_k c_k (n-1)^k (x fastest); node feature f_i = mean log kappa over the
// 2^d elements around node i.  Per column j of a residual block r:
//   q = D^-1 r_j, rho_j = sqrt(mean_i q_i^2), input channels (q / rho_j, f),
//   S(r)_j = rho_j * net(q / rho_j, f)        (zero when rho_j = 0).
// Convolution: y[b][co][i] = bias[co] + sum_ci sum_t W[co][ci][t] x[b][ci][i + o_t],
// tap t = sum_k (o_k + 1) 3^k.  Parameters are one flat float vector
// [W1, b1, W2, b2, W3, b3, W4, b4]; the network computes with the parameters rounded to
// bfloat16 and accumulates in FP32; Adam updates the FP32 master copy.
//
// Training loss per column (e = the error the solver's iterate carries, r = A e):
//   L = (e - S(r))^T A (e - S(r)) / (e^T r),
// the squared energy norm of the error left after one smoothing step relative to the
// error before it.  Its gradient with respect to the network output is
// -2 rho (A (e - S(r))) / (B e^T r) for a batch of B columns.
//
// Layout: activations [B][C][N] FP32 (nodes fastest, so neighbouring threads read
// neighbouring nodes); the residual / correction blocks stay node-major [N][m].
#include <cuda_bf16.h>

#include <algorithm>

#include "pase_internal.h"
#include "tc_util.h"

namespace pase {

constexpr int kSmC = 16;       // hidden channels
constexpr int kSmBatch = 8;    // columns per network pass
constexpr int kSmWgBlocks = 608;

template <int DIM>
struct Taps {
  static constexpr int T = DIM == 2 ? 9 : 27;
};

// interior-grid coordinates of node i
template <int DIM>
__device__ __forceinline__ void node_coords(int64_t i, int n1, int& cx, int& cy, int& cz) {
  cx = (int)(i % n1);
  const int64_t rest = i / n1;
  if (DIM == 2) {
    cy = (int)rest;
    cz = 0;
  } else {
    cy = (int)(rest % n1);
    cz = (int)(rest / n1);
  }
}

// ------------------------------------------------------------------ features, scaling
__global__ void k_sm_feat(int dim, int n, int n1, int64_t N, const double* __restrict__ logk, float* __restrict__ f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int cx = (int)(i % n1);
    const int64_t rest = i / n1;
    const int cy = (int)(rest % n1), cz = dim == 3 ? (int)(rest / n1) : 0;
    double s = 0.0;
    const int corners = 1 << dim;
    for (int q = 0; q < corners; ++q) {
      const int ex = cx + (q & 1), ey = cy + ((q >> 1) & 1), ez = dim == 3 ? cz + ((q >> 2) & 1) : 0;
      s += logk ? logk[(int64_t)ex + (int64_t)n * (ey + (int64_t)n * ez)] : 0.0;
    }
    f[i] = (float)(s / corners);
  }
}

// partial[blk][b] = sum over the block's rows of (dinv_i R[i][c0+b])^2, b < bc
template <typename T>
__global__ void __launch_bounds__(256) k_sm_colsq(int64_t N, int c0, int bc, const T* __restrict__ R, int64_t ldr,
                                                  const T* __restrict__ dinv, double* __restrict__ partial) {
  __shared__ double red[256];
  const int b = threadIdx.x % kSmBatch, g = threadIdx.x / kSmBatch;  // 32 row groups x 8 columns
  double s = 0.0;
  if (b < bc)
    for (int64_t i = (int64_t)blockIdx.x * 32 + g; i < N; i += (int64_t)gridDim.x * 32) {
      const double q = (double)dinv[i] * (double)R[i * ldr + c0 + b];
      s = fma(q, q, s);
    }
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < kSmBatch) {
    double t = 0.0;
    for (int q = 0; q < 32; ++q) t += red[q * kSmBatch + threadIdx.x];
    partial[(int64_t)blockIdx.x * kSmBatch + threadIdx.x] = t;
  }
}

// rho[b] = sqrt(sum[b] / N)
__global__ void k_sm_rho(int bc, int64_t N, const double* __restrict__ sums, double* __restrict__ rho) {
  const int b = threadIdx.x;
  if (b < bc) rho[b] = sqrt(sums[b] / (double)N);
}

// act0[b][0][i] = dinv_i R[i][c0+b] / rho_b, act0[b][1][i] = f_i
template <typename T>
__global__ void k_sm_gather(int64_t N, int c0, int bc, const T* __restrict__ R, int64_t ldr, const T* __restrict__ dinv,
                            const double* __restrict__ rho, const float* __restrict__ feat, float* __restrict__ act0) {
  const int b = blockIdx.y;
  const double rb = rho[b];
  const double inv = rb > 0.0 ? 1.0 / rb : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    act0[((int64_t)b * 2) * N + i] = (float)((double)dinv[i] * (double)R[i * ldr + c0 + b] * inv);
    act0[((int64_t)b * 2 + 1) * N + i] = feat[i];
  }
}

// ------------------------------------------------------------------ convolution
// Z[b][co][i] = bias[co] + sum_ci sum_t W[co][ci][t] act(X[b][ci][i + o_t]) (zero outside
// the grid); act = ReLU when relu_in, identity otherwise; the result is multiplied by
// [mask[b][co][i] > 0] when mask is given (backward pass through a ReLU).
template <int DIM, int CIN, int COUT>
__global__ void __launch_bounds__(256) k_sm_conv(int64_t N, int n1, const float* __restrict__ X, int relu_in,
                                                 const float* __restrict__ W, const float* __restrict__ bias,
                                                 const float* __restrict__ mask, float* __restrict__ Z) {
  constexpr int T = Taps<DIM>::T;
  __shared__ float ws[COUT * CIN * T + COUT];
  for (int k = threadIdx.x; k < COUT * CIN * T; k += blockDim.x) ws[k] = W[k];
  for (int k = threadIdx.x; k < COUT; k += blockDim.x) ws[COUT * CIN * T + k] = bias ? bias[k] : 0.f;
  __syncthreads();
  const int b = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int cx, cy, cz;
  node_coords<DIM>(i, n1, cx, cy, cz);
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = ws[COUT * CIN * T + co];
  const int64_t n1l = n1;
  for (int ci = 0; ci < CIN; ++ci) {
    const float* xb = X + ((int64_t)b * CIN + ci) * N;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int ox = t % 3 - 1, oy = (t / 3) % 3 - 1, oz = DIM == 3 ? t / 9 - 1 : 0;
      const bool ok = (unsigned)(cx + ox) < (unsigned)n1 && (unsigned)(cy + oy) < (unsigned)n1 &&
                      (DIM == 2 || (unsigned)(cz + oz) < (unsigned)n1);
      float v = ok ? xb[i + ox + oy * n1l + oz * n1l * n1l] : 0.f;
      if (relu_in) v = fmaxf(v, 0.f);
#pragma unroll
      for (int co = 0; co < COUT; ++co) acc[co] = fmaf(ws[(co * CIN + ci) * T + t], v, acc[co]);
    }
  }
#pragma unroll
  for (int co = 0; co < COUT; ++co) {
    float o = acc[co];
    const int64_t idx = ((int64_t)b * COUT + co) * N + i;
    if (mask && !(mask[idx] > 0.f)) o = 0.f;
    Z[idx] = o;
  }
}

// ------------------------------------------------------------------ inference path
// The V-cycle applies the network with its hidden activations stored in bfloat16,
// node-major [B][N][16] (32 bytes per node).  Layer 1 (2 -> 16) and layer 4 (16 -> 1) run
// on the CUDA cores; the two 16 -> 16 layers are implicit GEMMs on the tensor cores
// (tcgen05): per tile of 128 nodes, M = 128 nodes, N = 16 output channels, K = 16 input
// channels per tap, one MMA per tap accumulating in tensor memory.

// inference input: S[b][i] = dinv_i R[i][c0+b] / rho_b, one thread per node for all bc
// columns (contiguous reads of the node's row of R)
template <typename T>
__global__ void k_sm_gather_s(int64_t N, int c0, int bc, const T* __restrict__ R, int64_t ldr,
                              const T* __restrict__ dinv, const double* __restrict__ rho, float* __restrict__ S) {
  __shared__ double inv[kSmBatch];
  if (threadIdx.x < kSmBatch) inv[threadIdx.x] = (threadIdx.x < bc && rho[threadIdx.x] > 0.0) ? 1.0 / rho[threadIdx.x] : 0.0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double dv = (double)dinv[i];
    for (int b = 0; b < bc; ++b) S[(int64_t)b * N + i] = (float)(dv * (double)R[i * ldr + c0 + b] * inv[b]);
  }
}

constexpr int kTcTile = 128;                                      // nodes per MMA tile (M)
constexpr uint32_t kTcIdesc = umma_idesc_bf16(kTcTile, 16);       // M = 128, N = 16

// Tiles of 8 (x) x 16 (y) nodes (one z plane in 3D).  The tile's input halo (10 x 18
// nodes, times 3 z planes in 3D) is staged once in shared memory as two planes, channels
// 0-7 and channels 8-15, 16 bytes per node.  In the canonical K-major layout a core
// matrix is then 8 consecutive x nodes of one plane, the 16 groups of 8 rows are the 16
// halo rows (SBO = the halo row pitch) and the two K halves are the two planes (LBO =
// plane size), so the A operand of tap t is the same halo addressed from a start shifted
// by the tap's offset: no per-tap copies.
constexpr int kTcX = 8, kTcY = 16, kTcHX = kTcX + 2, kTcHY = kTcY + 2;
__host__ __device__ inline int tc_halo_nodes(int dim) { return kTcHX * kTcHY * (dim == 3 ? 3 : 1); }
__host__ __device__ inline size_t tc_smem_bytes(int dim) {
  const int T = dim == 2 ? 9 : 27;
  return (size_t)2 * tc_halo_nodes(dim) * 16 + (size_t)T * 512 + 256;
}

// LAYER 0: the 2 -> 16 input layer from S[b][N] (scaled residual) and f[N] (node
// feature), both rounded to bf16, the input channels padded to K = 16 with zeros;
// LAYER 1: a 16 -> 16 hidden layer; both give Y = bf16(ReLU(bias + conv)).
// LAYER 2: the 16 -> 1 output layer with the update fused, Xo[i][c0+b] (+)= rho_b
// (bias + conv(X)); the output channel is padded to N = 16 with zero weights.
template <int DIM, int LAYER, typename TO>
__global__ void __launch_bounds__(kTcTile) k_sm_conv_tc(int64_t N, int n1, int B, const __nv_bfloat16* __restrict__ X,
                                                        const float* __restrict__ S, const float* __restrict__ feat,
                                                        const float* __restrict__ W, const float* __restrict__ bias,
                                                        __nv_bfloat16* __restrict__ Y, int* __restrict__ err,
                                                        const double* __restrict__ rho, TO* __restrict__ Xo,
                                                        int64_t ldx, int c0, int add) {
  constexpr bool LAST = LAYER == 2;
  constexpr int T = Taps<DIM>::T;
  constexpr int HZ = DIM == 3 ? 3 : 1;
  constexpr int HN = kTcHX * kTcHY * HZ;  // halo nodes
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  uint4* plane0 = reinterpret_cast<uint4*>(tc_smem);                 // channels 0-7, [HZ][HY][HX]
  uint4* plane1 = plane0 + HN;                                        // channels 8-15
  __nv_bfloat16* sB = reinterpret_cast<__nv_bfloat16*>(tc_smem + (size_t)2 * HN * 16);  // [T][16 x 16]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float sbias[kSmC];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < T * 256; k += kTcTile) {
    const int t = k / 256, rem = k % 256, co = rem / 16, ci = rem % 16;
    float wv;
    if (LAYER == 0) wv = ci < 2 ? W[(co * 2 + ci) * T + t] : 0.f;
    else wv = (LAST && co > 0) ? 0.f : W[(co * kSmC + ci) * T + t];
    sB[t * 256 + (co / 8) * 128 + (ci / 8) * 64 + (co % 8) * 8 + (ci % 8)] = __float2bfloat16(wv);
  }
  if (tid < kSmC) sbias[tid] = (LAST && tid > 0) ? 0.f : bias[tid];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int ntx = (n1 + kTcX - 1) / kTcX, nty = (n1 + kTcY - 1) / kTcY, ntz = DIM == 3 ? n1 : 1;
  const int64_t tiles_per_col = (int64_t)ntx * nty * ntz;
  const int64_t ntiles = tiles_per_col * B;
  const int64_t n1l = n1;
  const uint32_t p0 = smem_u32(plane0);
  const uint32_t lbo = (uint32_t)HN * 16, sbo = kTcHX * 16;
  uint32_t phase = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int b = (int)(tile / tiles_per_col);
    int64_t rem = tile % tiles_per_col;
    const int tx = (int)(rem % ntx);
    rem /= ntx;
    const int ty = (int)(rem % nty);
    const int tz = (int)(rem / nty);
    const int x0 = tx * kTcX, y0 = ty * kTcY, z0 = tz;
    const __nv_bfloat16* Xb = X + (int64_t)b * N * kSmC;
    // stage the halo (zero outside the grid)
    for (int e = tid; e < HN; e += kTcTile) {
      const int hx = e % kTcHX, hy = (e / kTcHX) % kTcHY, hz = e / (kTcHX * kTcHY);
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = DIM == 3 ? z0 - 1 + hz : 0;
      uint4 lo = make_uint4(0, 0, 0, 0), hi = lo;
      if ((unsigned)gx < (unsigned)n1 && (unsigned)gy < (unsigned)n1 && (DIM == 2 || (unsigned)gz < (unsigned)n1)) {
        const int64_t node = gx + gy * n1l + gz * n1l * n1l;
        if (LAYER == 0) {
          __nv_bfloat162 sf = __floats2bfloat162_rn(S[(int64_t)b * N + node], feat[node]);
          lo.x = *reinterpret_cast<uint32_t*>(&sf);
        } else {
          const uint4* src = reinterpret_cast<const uint4*>(Xb + node * kSmC);
          lo = __ldg(src);
          hi = __ldg(src + 1);
        }
      }
      plane0[e] = lo;
      plane1[e] = hi;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      for (int t = 0; t < T; ++t) {
        const int ox = t % 3 - 1, oy = (t / 3) % 3 - 1, oz = DIM == 3 ? t / 9 - 1 : 0;
        const int base = ((DIM == 3 ? (1 + oz) : 0) * kTcHY + (1 + oy)) * kTcHX + (1 + ox);
        const uint64_t da = umma_desc(p0 + (uint32_t)base * 16, lbo, sbo);
        const uint64_t db = umma_desc(smem_u32(sB + t * 256), 128, 256);
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(kTcIdesc), "r"(t));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    const uint32_t done = mbar_wait_bounded(smem_u32(&mbar), phase, 1 << 22);
    if (!__syncthreads_and((int)done)) {  // (uniform) give up: report, let the MMAs finish, stop
      if (tid == 0) atomicExch(err, 1);
      mbar_wait_bounded(smem_u32(&mbar), phase, 1 << 22);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t r[16];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    // accumulator row = tid: node (x0 + tid % 8, y0 + tid / 8, z0)
    const int gx = x0 + (tid % kTcX), gy = y0 + (tid / kTcX);
    if (gx < n1 && gy < n1) {
      const int64_t node = gx + gy * n1l + (int64_t)z0 * n1l * n1l;
      if (LAST) {
        const double d = rho[b] * (double)(__uint_as_float(r[0]) + sbias[0]);
        TO* p = Xo + node * ldx + c0 + b;
        *p = add ? (TO)((double)*p + d) : (TO)d;
      } else {
        __align__(16) __nv_bfloat16 out[kSmC];
#pragma unroll
        for (int c = 0; c < kSmC; ++c) out[c] = __float2bfloat16(fmaxf(__uint_as_float(r[c]) + sbias[c], 0.f));
        uint4* dst = reinterpret_cast<uint4*>(Y + ((int64_t)b * N + node) * kSmC);
        dst[0] = reinterpret_cast<const uint4*>(out)[0];
        dst[1] = reinterpret_cast<const uint4*>(out)[1];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // the halo and the accumulator are reused by the next tile
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// Weight gradient of one layer: partial[blk][(co*CIN + ci)*T + t] = sum over the block's
// grid rows and all b of G[b][co][i] act(X[b][ci][i + o_t]); bias gradients after the
// weights (partial[blk][COUT*CIN*T + co] = sum G[b][co][i]).  A grid row is a run of n1
// nodes along x; the block's rows are [r0, r1).
template <int DIM, int CIN, int COUT>
__global__ void __launch_bounds__(256) k_sm_wgrad(int B, int64_t N, int n1, const float* __restrict__ X, int relu_in,
                                                  const float* __restrict__ G, int64_t rows_per_block,
                                                  double* __restrict__ partial) {
  constexpr int T = Taps<DIM>::T;
  constexpr int W = COUT * CIN * T + COUT;
  const int64_t nrows = N / n1;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < nrows ? r0 + rows_per_block : nrows;
  const int64_t n1l = n1;
  for (int it = threadIdx.x; it < COUT * T + COUT; it += blockDim.x) {
    if (it < COUT * T) {
      const int co = it / T, t = it % T;
      const int ox = t % 3 - 1, oy = (t / 3) % 3 - 1, oz = DIM == 3 ? t / 9 - 1 : 0;
      const int x0 = ox < 0 ? 1 : 0, x1 = ox > 0 ? n1 - 1 : n1;
      float acc[CIN];
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.f;
      for (int b = 0; b < B; ++b)
        for (int64_t row = r0; row < r1; ++row) {
          const int ry = DIM == 2 ? (int)row : (int)(row % n1);
          const int rz = DIM == 2 ? 0 : (int)(row / n1);
          if ((unsigned)(ry + oy) >= (unsigned)n1 || (DIM == 3 && (unsigned)(rz + oz) >= (unsigned)n1)) continue;
          const float* g = G + ((int64_t)b * COUT + co) * N + row * n1l;
          const int64_t shift = ox + oy * n1l + oz * n1l * n1l;
          for (int x = x0; x < x1; ++x) {
            const float gv = g[x];
            const int64_t src = row * n1l + x + shift;
#pragma unroll
            for (int ci = 0; ci < CIN; ++ci) {
              float v = X[((int64_t)b * CIN + ci) * N + src];
              if (relu_in) v = fmaxf(v, 0.f);
              acc[ci] = fmaf(gv, v, acc[ci]);
            }
          }
        }
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) partial[(int64_t)blockIdx.x * W + (co * CIN + ci) * T + t] = (double)acc[ci];
    } else {
      const int co = it - COUT * T;
      double s = 0.0;
      for (int b = 0; b < B; ++b) {
        const float* g = G + ((int64_t)b * COUT + co) * N;
        float a = 0.f;
        for (int64_t i = r0 * n1l; i < r1 * n1l; ++i) a += g[i];
        s += a;
      }
      partial[(int64_t)blockIdx.x * W + COUT * CIN * T + co] = s;
    }
  }
}

// Wt[(co'*CIN' + ci')*T + t] = W[(ci'*CIN + co')*T + (T-1-t)] with CIN' = COUT, COUT' = CIN:
// the weights of the transposed convolution (input gradient), taps mirrored.
__global__ void k_sm_transpose(int cin, int cout, int T, const float* __restrict__ W, float* __restrict__ Wt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cin * cout * T) return;
  const int t = k % T, rest = k / T;
  const int ci2 = rest % cout, co2 = rest / cout;  // Wt index (co2 in [0,cin), ci2 in [0,cout))
  Wt[k] = W[((int64_t)ci2 * cin + co2) * T + (T - 1 - t)];
}

// Adam on the FP32 master parameters; peff = the parameters rounded to bfloat16
__global__ void k_sm_adam(int P, const double* __restrict__ grad, float* __restrict__ p, float* __restrict__ m,
                          float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2,
                          float* __restrict__ peff) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const float g = (float)grad[k];
  const float mk = b1 * m[k] + (1.f - b1) * g;
  const float vk = b2 * v[k] + (1.f - b2) * g * g;
  m[k] = mk;
  v[k] = vk;
  const float pk = p[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
  p[k] = pk;
  peff[k] = __bfloat162float(__float2bfloat16_rn(pk));
}

__global__ void k_sm_round(int P, const float* __restrict__ p, float* __restrict__ peff) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < P) peff[k] = __bfloat162float(__float2bfloat16_rn(p[k]));
}

// E[i][b] = e[i][b] - rho_b y[b][i]   ([N][B] blocks, B = kSmBatch)
__global__ void k_sm_err(int64_t N, int B, const double* __restrict__ e, const float* __restrict__ y,
                         const double* __restrict__ rho, double* __restrict__ E) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N * B; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / B;
    const int b = (int)(k % B);
    E[k] = e[k] - rho[b] * (double)y[(int64_t)b * N + i];
  }
}

// gy[b][i] = -2 rho_b AE[i][b] / (B den_b)
__global__ void k_sm_outgrad(int64_t N, int B, const double* __restrict__ AE, const double* __restrict__ rho,
                             const double* __restrict__ den, float* __restrict__ gy) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N * B; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / B;
    const int b = (int)(k % B);
    gy[(int64_t)b * N + i] = (float)(-2.0 * rho[b] * AE[k] / ((double)B * den[b]));
  }
}

// E[i][b] = e[i][b] - omega dinv_i r[i][b]  (the damped Jacobi correction, for comparison)
__global__ void k_sm_jacobi_err(int64_t N, int B, const double* __restrict__ e, const double* __restrict__ r,
                                const double* __restrict__ dinv, double omega, double* __restrict__ E) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N * B; k += (int64_t)gridDim.x * blockDim.x)
    E[k] = e[k] - omega * dinv[k / B] * r[k];
}

static inline int sm_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------------ host side
struct LayerOff {
  int64_t W, b;
  int cin, cout;
};
static void layer_offsets(int T, LayerOff L[4]) {
  const int cin[4] = {2, kSmC, kSmC, kSmC}, cout[4] = {kSmC, kSmC, kSmC, 1};
  int64_t o = 0;
  for (int l = 0; l < 4; ++l) {
    L[l].cin = cin[l];
    L[l].cout = cout[l];
    L[l].W = o;
    o += (int64_t)cin[l] * cout[l] * T;
    L[l].b = o;
    o += cout[l];
  }
}

int smoother_nparams(int dim) {
  if (dim != 2 && dim != 3) return 0;
  const int T = dim == 2 ? 9 : 27;
  LayerOff L[4];
  layer_offsets(T, L);
  return (int)(L[3].b + 1);
}

bool sm_active(const pase_ctx* h) {
  return h->opt.smoother == PASE_SMOOTHER_LEARNED && h->sm && h->sm->has_params && !h->sm->rejected &&
         !h->sm_suspend && h->sm->N == h->N;
}

static int sm_check(pase_ctx* h) {
  if (!h->sm || h->sm->dim == 0) return fail(PASE_ERR_STATE, "learned smoother: pase_set_grid has not been called");
  return PASE_OK;
}

static int sync_stream(pase_ctx* h) {
  if (h->stream) PASE_CUDA(cudaStreamSynchronize(h->stream));
  else PASE_CUDA(cudaDeviceSynchronize());
  return PASE_OK;
}

int sm_set_grid(pase_ctx* h, int dim, int n, const double* logk_host) {
  if (dim != 2 && dim != 3) return fail(PASE_ERR_INVALID_ARG, "pase_set_grid: dim must be 2 or 3");
  if (n < 3) return fail(PASE_ERR_INVALID_ARG, "pase_set_grid: n must be at least 3");
  int64_t N = 1, ne = 1;
  for (int k = 0; k < dim; ++k) {
    N *= (n - 1);
    ne *= n;
  }
  if (N != h->N) return fail(PASE_ERR_SHAPE_MISMATCH, "pase_set_grid: (n-1)^dim differs from the fine level size");
  if (h->sm) return fail(PASE_ERR_STATE, "pase_set_grid: the grid is already set");
  Smoother* s = new (std::nothrow) Smoother();
  if (!s) return fail(PASE_ERR_OUT_OF_MEMORY, "pase_set_grid: host allocation");
  h->sm = s;
  s->dim = dim;
  s->n = n;
  s->n1 = n - 1;
  s->N = N;
  s->T = dim == 2 ? 9 : 27;
  s->P = smoother_nparams(dim);
  const int64_t NB = N * kSmBatch;
  PASE_TRY(dev_alloc_t(h, &s->feat, N));
  PASE_TRY(dev_alloc_t(h, &s->params, s->P));
  PASE_TRY(dev_alloc_t(h, &s->adam_m, s->P));
  PASE_TRY(dev_alloc_t(h, &s->adam_v, s->P));
  PASE_TRY(dev_alloc_t(h, &s->peff, s->P));
  PASE_TRY(dev_alloc_t(h, &s->wt, kSmC * kSmC * 27));
  PASE_TRY(dev_alloc_t(h, &s->grad, s->P));
  PASE_TRY(dev_alloc_t(h, &s->partial, (int64_t)kSmWgBlocks * (kSmC * kSmC * 27 + kSmC)));
  PASE_TRY(dev_alloc_t(h, &s->colpart, (int64_t)kReduceBlocksHost * kSmBatch));
  PASE_TRY(dev_alloc_t(h, &s->act0, 2 * NB));
  PASE_TRY(dev_alloc_t(h, &s->z1, kSmC * NB));
  PASE_TRY(dev_alloc_t(h, &s->z2, kSmC * NB));
  PASE_TRY(dev_alloc_t(h, &s->z3, kSmC * NB));
  PASE_TRY(dev_alloc_t(h, &s->y, NB));
  PASE_TRY(dev_alloc_t(h, &s->ga, kSmC * NB));
  PASE_TRY(dev_alloc_t(h, &s->gb, kSmC * NB));
  PASE_TRY(dev_alloc_t(h, &s->E, NB));
  PASE_TRY(dev_alloc_t(h, &s->AE, NB));
  PASE_TRY(dev_alloc_t(h, &s->e, NB));
  PASE_TRY(dev_alloc_t(h, &s->r, NB));
  PASE_TRY(dev_alloc_t(h, &s->sums, 8 * kSmBatch));
  PASE_TRY(dev_alloc_t(h, &s->tc_err, 1));
  PASE_CUDA(cudaMemsetAsync(s->tc_err, 0, sizeof(int), h->stream));
  PASE_CUDA(cudaMallocHost(&s->h_sums, sizeof(double) * 8 * kSmBatch));
  double* dl = nullptr;
  if (logk_host) {
    PASE_TRY(dev_alloc_t(h, &dl, ne));
    PASE_CUDA(cudaMemcpyAsync(dl, logk_host, sizeof(double) * ne, cudaMemcpyHostToDevice, h->stream));
  }
  k_sm_feat<<<sm_grid(N), 256, 0, h->stream>>>(dim, n, n - 1, N, dl, s->feat);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  PASE_CUDA(cudaMemsetAsync(s->params, 0, sizeof(float) * s->P, h->stream));
  PASE_CUDA(cudaMemsetAsync(s->peff, 0, sizeof(float) * s->P, h->stream));
  PASE_CUDA(cudaMemsetAsync(s->adam_m, 0, sizeof(float) * s->P, h->stream));
  PASE_CUDA(cudaMemsetAsync(s->adam_v, 0, sizeof(float) * s->P, h->stream));
  return sync_stream(h);
}

// state = [params | adam m | adam v | t] (3P + 1 floats, host memory)
int sm_state(pase_ctx* h, float* buf, int64_t count, bool get) {
  PASE_TRY(sm_check(h));
  Smoother* s = h->sm;
  if (count != 3 * (int64_t)s->P + 1) return fail(PASE_ERR_INVALID_ARG, "smoother state: count must be 3P + 1");
  if (!buf) return fail(PASE_ERR_INVALID_ARG, "smoother state: null buffer");
  if (get) {
    PASE_CUDA(cudaMemcpyAsync(buf, s->params, sizeof(float) * s->P, cudaMemcpyDeviceToHost, h->stream));
    PASE_CUDA(cudaMemcpyAsync(buf + s->P, s->adam_m, sizeof(float) * s->P, cudaMemcpyDeviceToHost, h->stream));
    PASE_CUDA(cudaMemcpyAsync(buf + 2 * s->P, s->adam_v, sizeof(float) * s->P, cudaMemcpyDeviceToHost, h->stream));
    PASE_TRY(sync_stream(h));
    buf[3 * s->P] = (float)s->t;
    return PASE_OK;
  }
  for (int64_t k = 0; k < count; ++k)
    if (!isfinite(buf[k])) return fail(PASE_ERR_NAN, "smoother state: non-finite value");
  if (buf[3 * s->P] < 0.f) return fail(PASE_ERR_INVALID_ARG, "smoother state: negative step count");
  PASE_CUDA(cudaMemcpyAsync(s->params, buf, sizeof(float) * s->P, cudaMemcpyHostToDevice, h->stream));
  PASE_CUDA(cudaMemcpyAsync(s->adam_m, buf + s->P, sizeof(float) * s->P, cudaMemcpyHostToDevice, h->stream));
  PASE_CUDA(cudaMemcpyAsync(s->adam_v, buf + 2 * s->P, sizeof(float) * s->P, cudaMemcpyHostToDevice, h->stream));
  k_sm_round<<<(s->P + 255) / 256, 256, 0, h->stream>>>(s->P, s->params, s->peff);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  PASE_TRY(sync_stream(h));
  s->t = (int)buf[3 * s->P];
  s->has_params = true;
  s->rejected = false;
  return PASE_OK;
}

template <int DIM, int CIN, int COUT>
static int conv_launch(pase_ctx* h, int B, const float* X, int relu_in, const float* W, const float* bias,
                       const float* mask, float* Z) {
  const Smoother* s = h->sm;
  dim3 grid((unsigned)((s->N + 255) / 256), (unsigned)B);
  k_sm_conv<DIM, CIN, COUT><<<grid, 256, 0, h->stream>>>(s->N, s->n1, X, relu_in, W, bias, mask, Z);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

template <int DIM>
static int forward(pase_ctx* h, int B) {
  Smoother* s = h->sm;
  LayerOff L[4];
  layer_offsets(s->T, L);
  const float* p = s->peff;
  PASE_TRY((conv_launch<DIM, 2, kSmC>(h, B, s->act0, 0, p + L[0].W, p + L[0].b, nullptr, s->z1)));
  PASE_TRY((conv_launch<DIM, kSmC, kSmC>(h, B, s->z1, 1, p + L[1].W, p + L[1].b, nullptr, s->z2)));
  PASE_TRY((conv_launch<DIM, kSmC, kSmC>(h, B, s->z2, 1, p + L[2].W, p + L[2].b, nullptr, s->z3)));
  PASE_TRY((conv_launch<DIM, kSmC, 1>(h, B, s->z3, 1, p + L[3].W, p + L[3].b, nullptr, s->y)));
  return PASE_OK;
}

// inference pass for columns c0..c0+bc-1 of R: X (+)= S(R) (bf16 hidden activations,
// tensor-core hidden layers); rho must already be in sums[kSmBatch..]
template <int DIM, typename T>
static int forward_fast(pase_ctx* h, int c0, int bc, const T* R, int64_t ldr, const T* dinv, T* X, int64_t ldx,
                        bool add) {
  Smoother* s = h->sm;
  LayerOff L[4];
  layer_offsets(s->T, L);
  const float* p = s->peff;
  const double* rho = s->sums + kSmBatch;
  __nv_bfloat16* y1 = reinterpret_cast<__nv_bfloat16*>(s->z1);
  __nv_bfloat16* y2 = reinterpret_cast<__nv_bfloat16*>(s->z2);
  const int gn = (int)std::min<int64_t>((s->N + 255) / 256, 4096);
  k_sm_gather_s<T><<<gn, 256, 0, h->stream>>>(s->N, c0, bc, R, ldr, dinv, rho, s->act0);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  const size_t smem = tc_smem_bytes(DIM);
  PASE_TRY(ensure_max_smem((const void*)k_sm_conv_tc<DIM, 0, T>, 200 * 1024));
  PASE_TRY(ensure_max_smem((const void*)k_sm_conv_tc<DIM, 1, T>, 200 * 1024));
  PASE_TRY(ensure_max_smem((const void*)k_sm_conv_tc<DIM, 2, T>, 200 * 1024));
  const int64_t tiles = (int64_t)((s->n1 + kTcX - 1) / kTcX) * ((s->n1 + kTcY - 1) / kTcY) *
                        (DIM == 3 ? s->n1 : 1) * bc;
  const int per_sm = std::max(1, (int)((220 * 1024) / (smem + 1024)));
  const int tcgrid = (int)std::min<int64_t>(tiles, (int64_t)152 * per_sm);
  k_sm_conv_tc<DIM, 0, T><<<tcgrid, kTcTile, smem, h->stream>>>(s->N, s->n1, bc, nullptr, s->act0, s->feat, p + L[0].W,
                                                                p + L[0].b, y1, s->tc_err, nullptr, nullptr, 0, 0, 0);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  k_sm_conv_tc<DIM, 1, T><<<tcgrid, kTcTile, smem, h->stream>>>(s->N, s->n1, bc, y1, nullptr, nullptr, p + L[1].W,
                                                                p + L[1].b, y2, s->tc_err, nullptr, nullptr, 0, 0, 0);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  k_sm_conv_tc<DIM, 1, T><<<tcgrid, kTcTile, smem, h->stream>>>(s->N, s->n1, bc, y2, nullptr, nullptr, p + L[2].W,
                                                                p + L[2].b, y1, s->tc_err, nullptr, nullptr, 0, 0, 0);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  k_sm_conv_tc<DIM, 2, T><<<tcgrid, kTcTile, smem, h->stream>>>(s->N, s->n1, bc, y1, nullptr, nullptr, p + L[3].W,
                                                                p + L[3].b, nullptr, s->tc_err, rho, X, ldx, c0,
                                                                add ? 1 : 0);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// column sums of (D^-1 R)^2 and rho for columns c0..c0+bc-1 (into sums[kSmBatch..])
template <typename T>
static int scale_only(pase_ctx* h, int c0, int bc, const T* R, int64_t ldr, const T* dinv) {
  Smoother* s = h->sm;
  int64_t g = (s->N + 31) / 32;
  if (g > kReduceBlocksHost) g = kReduceBlocksHost;
  k_sm_colsq<T><<<(unsigned)g, 256, 0, h->stream>>>(s->N, c0, bc, R, ldr, dinv, s->colpart);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  PASE_TRY(launch_reduce_partials(h, (int)g, kSmBatch, s->colpart, s->sums));
  k_sm_rho<<<1, 32, 0, h->stream>>>(bc, s->N, s->sums, s->sums + kSmBatch);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

int sm_check_timeout(pase_ctx* h) {
  if (!h->sm || !h->sm->tc_err) return PASE_OK;
  int e = 0;
  PASE_CUDA(cudaMemcpyAsync(&e, h->sm->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PASE_TRY(sync_stream(h));
  if (e) {
    PASE_CUDA(cudaMemsetAsync(h->sm->tc_err, 0, sizeof(int), h->stream));
    return fail(PASE_ERR_TIMEOUT, "learned smoother: a tensor-core wait ran out of its limit");
  }
  return PASE_OK;
}

template <typename T>
static int normalise(pase_ctx* h, int c0, int bc, const T* R, int64_t ldr, const T* dinv) {
  Smoother* s = h->sm;
  int64_t g = (s->N + 31) / 32;
  if (g > kReduceBlocksHost) g = kReduceBlocksHost;
  k_sm_colsq<T><<<(unsigned)g, 256, 0, h->stream>>>(s->N, c0, bc, R, ldr, dinv, s->colpart);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  PASE_TRY(launch_reduce_partials(h, (int)g, kSmBatch, s->colpart, s->sums));
  k_sm_rho<<<1, 32, 0, h->stream>>>(bc, s->N, s->sums, s->sums + kSmBatch);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  dim3 grid((unsigned)std::min<int64_t>((s->N + 255) / 256, 1024), (unsigned)bc);
  k_sm_gather<T><<<grid, 256, 0, h->stream>>>(s->N, c0, bc, R, ldr, dinv, s->sums + kSmBatch, s->feat, s->act0);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

// X (+)= S(R) column block by column block (kSmBatch columns per pass)
template <typename T>
int sm_apply(pase_ctx* h, int m, const T* R, int64_t ldr, const T* dinv, T* X, int64_t ldx, bool add) {
  PASE_TRY(sm_check(h));
  Smoother* s = h->sm;
  for (int c0 = 0; c0 < m; c0 += kSmBatch) {
    const int bc = std::min(kSmBatch, m - c0);
    PASE_TRY(scale_only<T>(h, c0, bc, R, ldr, dinv));
    if (s->dim == 2) PASE_TRY((forward_fast<2, T>(h, c0, bc, R, ldr, dinv, X, ldx, add)));
    else PASE_TRY((forward_fast<3, T>(h, c0, bc, R, ldr, dinv, X, ldx, add)));
  }
  return PASE_OK;
}
template int sm_apply<double>(pase_ctx*, int, const double*, int64_t, const double*, double*, int64_t, bool);
template int sm_apply<float>(pase_ctx*, int, const float*, int64_t, const float*, float*, int64_t, bool);

template <int DIM, int CIN, int COUT>
static int wgrad_launch(pase_ctx* h, int B, const float* X, int relu_in, const float* G, double* grad_out) {
  Smoother* s = h->sm;
  const int64_t nrows = s->N / s->n1;
  int nblk = (int)std::min<int64_t>(nrows, kSmWgBlocks);
  const int64_t rpb = (nrows + nblk - 1) / nblk;
  nblk = (int)((nrows + rpb - 1) / rpb);
  k_sm_wgrad<DIM, CIN, COUT><<<nblk, 256, 0, h->stream>>>(B, s->N, s->n1, X, relu_in, G, rpb, s->partial);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  constexpr int T = Taps<DIM>::T;
  return launch_reduce_partials(h, nblk, COUT * CIN * T + COUT, s->partial, grad_out);
}

static int transpose_launch(pase_ctx* h, int cin, int cout, const float* W) {
  const int T = h->sm->T;
  const int n = cin * cout * T;
  k_sm_transpose<<<(n + 255) / 256, 256, 0, h->stream>>>(cin, cout, T, W, h->sm->wt);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

template <int DIM>
static int backward(pase_ctx* h, int B) {
  Smoother* s = h->sm;
  LayerOff L[4];
  layer_offsets(s->T, L);
  const float* p = s->peff;
  // layer 4: input relu(z3); the output gradient gy sits in the first N*B floats of gb
  float* gy = s->gb;
  PASE_TRY((wgrad_launch<DIM, kSmC, 1>(h, B, s->z3, 1, gy, s->grad + L[3].W)));
  PASE_TRY(transpose_launch(h, kSmC, 1, p + L[3].W));
  PASE_TRY((conv_launch<DIM, 1, kSmC>(h, B, gy, 0, s->wt, nullptr, s->z3, s->ga)));
  // layer 3
  PASE_TRY((wgrad_launch<DIM, kSmC, kSmC>(h, B, s->z2, 1, s->ga, s->grad + L[2].W)));
  PASE_TRY(transpose_launch(h, kSmC, kSmC, p + L[2].W));
  PASE_TRY((conv_launch<DIM, kSmC, kSmC>(h, B, s->ga, 0, s->wt, nullptr, s->z2, s->gb)));
  // layer 2
  PASE_TRY((wgrad_launch<DIM, kSmC, kSmC>(h, B, s->z1, 1, s->gb, s->grad + L[1].W)));
  PASE_TRY(transpose_launch(h, kSmC, kSmC, p + L[1].W));
  PASE_TRY((conv_launch<DIM, kSmC, kSmC>(h, B, s->gb, 0, s->wt, nullptr, s->z1, s->ga)));
  // layer 1 (input: the normalised residual and the feature)
  PASE_TRY((wgrad_launch<DIM, 2, kSmC>(h, B, s->act0, 0, s->ga, s->grad + L[0].W)));
  return PASE_OK;
}

// One training step on a batch of kSmBatch columns: e, r [N][B] device (r = A e).
// Writes the per-column losses (host, B doubles) and, if update, one Adam step.
int sm_step(pase_ctx* h, const double* e, const double* r, bool update, float lr, float b1, float b2, float eps,
            double* loss_cols) {
  PASE_TRY(sm_check(h));
  Smoother* s = h->sm;
  const int B = kSmBatch;
  const int64_t N = s->N;
  const DevCSR& A = h->lv[0].A;
  PASE_TRY(normalise<double>(h, 0, B, r, B, h->lv[0].dinv));
  if (s->dim == 2) PASE_TRY(forward<2>(h, B));
  else PASE_TRY(forward<3>(h, B));
  double* rho = s->sums + kSmBatch;
  double* num = s->sums + 2 * kSmBatch;
  double* den = s->sums + 3 * kSmBatch;
  k_sm_err<<<sm_grid(N * B), 256, 0, h->stream>>>(N, B, e, s->y, rho, s->E);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  PASE_TRY(launch_csr<double>(h, CSR_MV, B, A, A.val, nullptr, s->E, nullptr, nullptr, nullptr, nullptr, 0.0, s->AE,
                              nullptr, nullptr, nullptr));
  PASE_TRY(launch_coldot(h, N, B, s->E, s->AE, num));
  PASE_TRY(launch_coldot(h, N, B, e, r, den));
  k_sm_outgrad<<<sm_grid(N * B), 256, 0, h->stream>>>(N, B, s->AE, rho, den, s->gb);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  if (s->dim == 2) PASE_TRY(backward<2>(h, B));
  else PASE_TRY(backward<3>(h, B));
  if (update) {
    s->t += 1;
    const float bc1 = (float)(1.0 - pow((double)b1, (double)s->t));
    const float bc2 = (float)(1.0 - pow((double)b2, (double)s->t));
    k_sm_adam<<<(s->P + 255) / 256, 256, 0, h->stream>>>(s->P, s->grad, s->params, s->adam_m, s->adam_v, lr, b1, b2,
                                                          eps, bc1, bc2, s->peff);
    h->launches++;
    PASE_CUDA(cudaGetLastError());
  }
  PASE_CUDA(cudaMemcpyAsync(s->h_sums, num, sizeof(double) * 2 * kSmBatch, cudaMemcpyDeviceToHost, h->stream));
  PASE_TRY(sync_stream(h));
  for (int b = 0; b < B; ++b) loss_cols[b] = s->h_sums[b] / s->h_sums[kSmBatch + b];
  return PASE_OK;
}

// Energy loss of the damped Jacobi correction omega D^-1 r on the same kind of batch
int sm_jacobi_loss(pase_ctx* h, const double* e, const double* r, double* loss_cols) {
  PASE_TRY(sm_check(h));
  Smoother* s = h->sm;
  const int B = kSmBatch;
  const int64_t N = s->N;
  const DevCSR& A = h->lv[0].A;
  double* num = s->sums + 2 * kSmBatch;
  double* den = s->sums + 3 * kSmBatch;
  k_sm_jacobi_err<<<sm_grid(N * B), 256, 0, h->stream>>>(N, B, e, r, h->lv[0].dinv, h->opt.omega, s->E);
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  PASE_TRY(launch_csr<double>(h, CSR_MV, B, A, A.val, nullptr, s->E, nullptr, nullptr, nullptr, nullptr, 0.0, s->AE,
                              nullptr, nullptr, nullptr));
  PASE_TRY(launch_coldot(h, N, B, s->E, s->AE, num));
  PASE_TRY(launch_coldot(h, N, B, e, r, den));
  PASE_CUDA(cudaMemcpyAsync(s->h_sums, num, sizeof(double) * 2 * kSmBatch, cudaMemcpyDeviceToHost, h->stream));
  PASE_TRY(sync_stream(h));
  for (int b = 0; b < B; ++b) loss_cols[b] = s->h_sums[b] / s->h_sums[kSmBatch + b];
  return PASE_OK;
}

int sm_grad_to_host(pase_ctx* h, double* grad_host) {
  PASE_TRY(sm_check(h));
  PASE_CUDA(cudaMemcpyAsync(grad_host, h->sm->grad, sizeof(double) * h->sm->P, cudaMemcpyDeviceToHost, h->stream));
  return sync_stream(h);
}

void sm_free(pase_ctx* h) {
  if (h->sm) {
    if (h->sm->h_sums) cudaFreeHost(h->sm->h_sums);
    delete h->sm;
    h->sm = nullptr;
  }
}

}  // namespace pase
