// Structured-grid kernels of the FP32 smoothing path (damped-Jacobi sweep, residual,
// product) for operators that couple each node only to its 3^d grid neighbours.
//
// The step-(a) linear solve (Alg. 1 first step; Alg. 3 step 3) spends its time in damped
// Jacobi sweeps x <- x + omega D^-1 (b - A x) and residuals b - A x on the multigrid
// levels.  A Q1 operator on a uniform (n-1)^d interior grid with x-fastest ordering, and
// every Galerkin coarse operator of nested Q1 spaces, couples node (x, y, z) only to
// (x+dx, y+dy, z+dz) with |dx|, |dy|, |dz| <= 1, so its matrix needs no column indices.
//
// Why not the CSR kernel: with node-major multivectors [N][m] the CSR kernel gathers the
// m-wide X row of every nonzero through L1, 27 times per row in 3D, and the L1 request
// rate, not HBM, bounds it.
//
// Scheme.  A CTA owns a tile of the grid (16 x 4 nodes of an x-y plane in 3D, 64 nodes of
// an x line in 2D) and marches along the last axis (z in 3D, y in 2D) over a chunk of
// planes.  Plane p of X (the tile plus a one-node halo), the coefficients that meet it and
// b of plane p-1 arrive in shared memory by bulk asynchronous copies (cp.async.bulk,
// completion counted on an mbarrier), several planes ahead of the computation, in a ring
// of stages.  A thread owns 4 consecutive x rows and one 16-byte column slice; X values of
// plane p feed the three output planes p-1, p, p+1 through three rolling register
// accumulators, so each X value is read from shared memory once per (line, x window).  The
// damped-Jacobi sweep runs on the coefficients of its iteration matrix J = I - omega D^-1 A
// (y = J x + omega D^-1 b), so no copy of the old x is held for the update.  Every operand
// stream (X, b, coefficients, y) crosses HBM once.
//
// Coefficient layout ("step-major"), built at setup: the coefficient of row q's tap
// t = (dx+1) + 3(dy+1) + 9(dz+1) (2D: (dx+1) + 3(dy+1), dy the marching offset) is needed
// while plane q + dz is staged, so it is stored with step s = q + dz + 1, tile-blocked:
//   [s = 0 .. n1+1][tile y][tile x][slot 0 .. T][TY][TX]   (zeros outside the grid)
// slot T holding 1 / a_qq for plane q = s - 2 (the plane whose sweep completes then).  One
// bulk copy of (T+1) TY TX floats per tile and step.  A second array in the same layout
// holds J's coefficients (1 - omega a_qq / a_qq on the centre tap, -omega a_qj / a_qq
// elsewhere) with omega / a_qq in slot T, for the handle's omega.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "pase_internal.h"
#include "tc_util.h"

namespace pase {

namespace {

constexpr int kStMaxStages = 8;
constexpr int kStWaitLimit = 1 << 24;  // polls of a stage's mbarrier before giving up

template <int DIM>
struct StGeo {
  static constexpr int T = DIM == 3 ? 27 : 9;  // taps
  static constexpr int TX = DIM == 3 ? 16 : 64;
  static constexpr int TY = DIM == 3 ? 4 : 1;
  static constexpr int RUNS = TX / 4;               // 4-row x runs per tile line
  static constexpr int G = RUNS * TY;               // thread groups (16)
  static constexpr int NL = DIM == 3 ? TY + 2 : 1;  // staged X lines (halo included)
  static constexpr int VF = (T + 1) * TY * TX;      // coefficient floats per tile and step
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void fma4(float4& a, float s, const float4& x) {
  a.x = fmaf(s, x.x, a.x);
  a.y = fmaf(s, x.y, a.y);
  a.z = fmaf(s, x.z, a.z);
  a.w = fmaf(s, x.w, a.w);
}
// a consumer thread's column slice: 4 (float4) or 2 (float2) columns
template <int CW>
struct StVec;
template <>
struct StVec<4> {
  using T = float4;
  static __device__ __forceinline__ T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ T ld(const float* p) { return *reinterpret_cast<const float4*>(p); }
  static __device__ __forceinline__ void st(float* p, const T& v) { *reinterpret_cast<float4*>(p) = v; }
  static __device__ __forceinline__ void fma(T& a, float s, const T& x) { fma4(a, s, x); }
  static __device__ __forceinline__ T sub(const T& b, const T& o) {
    return make_float4(b.x - o.x, b.y - o.y, b.z - o.z, b.w - o.w);
  }
  static __device__ __forceinline__ T axpy(float d, const T& o, const T& x) {  // d o + x
    return make_float4(fmaf(d, o.x, x.x), fmaf(d, o.y, x.y), fmaf(d, o.z, x.z), fmaf(d, o.w, x.w));
  }
};
template <>
struct StVec<2> {
  using T = float2;
  static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ T ld(const float* p) { return *reinterpret_cast<const float2*>(p); }
  static __device__ __forceinline__ void st(float* p, const T& v) { *reinterpret_cast<float2*>(p) = v; }
  static __device__ __forceinline__ void fma(T& a, float s, const T& x) {
    a.x = fmaf(s, x.x, a.x);
    a.y = fmaf(s, x.y, a.y);
  }
  static __device__ __forceinline__ T sub(const T& b, const T& o) { return make_float2(b.x - o.x, b.y - o.y); }
  static __device__ __forceinline__ T axpy(float d, const T& o, const T& x) {
    return make_float2(fmaf(d, o.x, x.x), fmaf(d, o.y, x.y));
  }
};
__device__ __forceinline__ float vcomp(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// One staged plane, filled by the producer warp: the tile's X lines (halo included), the
// step's coefficients and (RESID, JACOBI) b of plane p-1, the plane whose update completes
// while this stage is current.  Lanes zero-fill the out-of-grid parts of the X lines, then
// lane 0 posts the expected byte count and lanes 0..(copies-1) issue one bulk copy each.
template <int DIM, bool WITH_B>
__device__ __forceinline__ void stage_fill(int lane, int n1, int m, int x0t, int y0t, int p, int64_t vblk,
                                           const float* __restrict__ X, const float* __restrict__ V,
                                           const float* __restrict__ B, float* xs, float* vs, float* bs,
                                           uint32_t full) {
  using Gm = StGeo<DIM>;
  const int64_t n1l = n1;
  const bool have_x = p >= 0 && p < n1;
  const bool have_b = WITH_B && p - 1 >= 0 && p - 1 < n1;
  const int xa = max(0, x0t - 1), xb = min(n1, x0t + Gm::TX + 1);  // in-grid node range of a line
  const int bxb = min(n1, x0t + Gm::TX);
  const bool interior = x0t >= 1 && x0t + Gm::TX + 1 <= n1 && (DIM == 2 || (y0t >= 1 && y0t + Gm::TY + 1 <= n1));
  if (have_x && !interior) {
    const int m4 = m / 4;
    for (int ly = 0; ly < Gm::NL; ++ly) {
      const int y = DIM == 3 ? y0t - 1 + ly : 0;
      const bool yok = DIM == 2 || (unsigned)y < (unsigned)n1;
      const int lo = yok ? xa - (x0t - 1) : Gm::TX + 2;  // nodes [0, lo) and [hi, TX+2) lie outside
      const int hi = yok ? xb - (x0t - 1) : Gm::TX + 2;
      const int nz = lo + (Gm::TX + 2 - hi);
      float4* line = reinterpret_cast<float4*>(xs + (int64_t)ly * (Gm::TX + 2) * m);
      for (int k = lane; k < nz * m4; k += 32) {
        const int zn = k / m4, c = k - zn * m4;
        line[(zn < lo ? zn : hi + (zn - lo)) * m4 + c] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  __syncwarp();
  // copy j: 0 = coefficients, 1..NL = X lines, NL+1..NL+TY = b lines (absent ones skipped)
  uint32_t bytes = (uint32_t)Gm::VF * 4u;
  if (have_x)
    for (int ly = 0; ly < Gm::NL; ++ly) {
      const int y = DIM == 3 ? y0t - 1 + ly : 0;
      if (DIM == 2 || (unsigned)y < (unsigned)n1) bytes += (uint32_t)(xb - xa) * (uint32_t)m * 4u;
    }
  if (have_b)
    for (int ly = 0; ly < Gm::TY; ++ly)
      if (DIM == 2 || y0t + ly < n1) bytes += (uint32_t)(bxb - x0t) * (uint32_t)m * 4u;
  if (lane == 0) asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full), "r"(bytes) : "memory");
  __syncwarp();
  if (lane == 0) bulk_g2s(smem_u32(vs), V + vblk, (uint32_t)Gm::VF * 4u, full);
  if (have_x && lane >= 1 && lane <= Gm::NL) {
    const int ly = lane - 1;
    const int y = DIM == 3 ? y0t - 1 + ly : 0;
    if (DIM == 2 || (unsigned)y < (unsigned)n1) {
      const int64_t node0 = DIM == 3 ? ((int64_t)p * n1l + y) * n1l + xa : (int64_t)p * n1l + xa;
      float* dst = xs + ((int64_t)ly * (Gm::TX + 2) + (xa - (x0t - 1))) * m;
      bulk_g2s(smem_u32(dst), X + node0 * m, (uint32_t)(xb - xa) * (uint32_t)m * 4u, full);
    }
  }
  if (have_b && lane > Gm::NL && lane <= Gm::NL + Gm::TY) {
    const int ly = lane - Gm::NL - 1;
    const int y = DIM == 3 ? y0t + ly : 0;
    if (DIM == 2 || y < n1) {
      const int64_t node0 = DIM == 3 ? ((int64_t)(p - 1) * n1l + y) * n1l + x0t : (int64_t)(p - 1) * n1l + x0t;
      bulk_g2s(smem_u32(bs + (int64_t)ly * Gm::TX * m), B + node0 * m, (uint32_t)(bxb - x0t) * (uint32_t)m * 4u, full);
    }
  }
}

// MODE: CSR_MV (y = A x), CSR_RESID (y = b - A x), CSR_JACOBI (y = x + omega dinv (b - A x)).
// Warp roles: the last warp fills stages (producer); the others compute (consumers).  A
// stage is filled once its "empty" barrier shows that every consumer warp has released its
// previous plane, and read once its "full" barrier shows the copies landed; no CTA-wide
// barrier in the loop, so consumer warps never wait for each other.
// CW: columns per consumer thread (4, or 2 for twice the threads at half the registers).
// MAXT, MINB: launch bounds - (256, 2) and (512, 1) give 128 registers per thread,
// (512, 2) 64.
template <int DIM, int MODE, int CW, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
    k_stencil(int n1, int m, int tpr, int ntx, int nty, int pch, int npc, int NS, const float* __restrict__ V,
              const float* __restrict__ X, const float* __restrict__ B, float omega, float* __restrict__ Y,
              int* __restrict__ err) {
  using Gm = StGeo<DIM>;
  using SV = StVec<CW>;
  using VT = typename SV::T;
  constexpr int T = Gm::T;
  constexpr bool WB = MODE == CSR_RESID || MODE == CSR_JACOBI;
  extern __shared__ __align__(128) float st_smem[];
  __shared__ __align__(8) uint64_t full[kStMaxStages], empty[kStMaxStages];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5, ncons = nwarps - 1;  // consumer warps
  const bool producer = warp == ncons;
  const int64_t xs_floats = (int64_t)Gm::NL * (Gm::TX + 2) * m;
  const int64_t bs_floats = WB ? (int64_t)Gm::TY * Gm::TX * m : 0;
  float* xs_base = st_smem;
  float* vs_base = st_smem + NS * xs_floats;
  float* bs_base = vs_base + (int64_t)NS * Gm::VF;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(ncons));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  __syncthreads();
  const int64_t n1l = n1;
  const int64_t items = (int64_t)ntx * nty * npc;
  int64_t gstep = 0;  // stage uses so far (ring position and barrier parities)
  if (producer) {
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
      const int tx = (int)(item % ntx);
      const int64_t r = item / ntx;
      const int ty = (int)(r % nty);
      const int pc = (int)(r / nty);
      const int x0t = tx * Gm::TX, y0t = ty * Gm::TY;
      const int pb = pc * pch, pe = min(n1, pb + pch);
      for (int p = pb - 1; p <= pe; ++p, ++gstep) {
        const int s = (int)(gstep % NS);
        if (gstep >= NS) {  // every consumer warp has released the plane this stage held
          const uint32_t ok = mbar_wait_bounded(smem_u32(&empty[s]), (uint32_t)((gstep / NS - 1) & 1), kStWaitLimit);
          if (!__all_sync(0xffffffffu, ok) || *(volatile int*)&abort_flag) {
            if (lane == 0) {
              atomicExch(err, 1);
              *(volatile int*)&abort_flag = 1;
            }
            item = items;
            break;
          }
        }
        const int64_t vblk = (((int64_t)(p + 1) * nty + ty) * ntx + tx) * Gm::VF;
        stage_fill<DIM, WB>(lane, n1, m, x0t, y0t, p, vblk, X, V, B, xs_base + s * xs_floats,
                            vs_base + (int64_t)s * Gm::VF, bs_base + s * bs_floats, smem_u32(&full[s]));
      }
    }
    // let the copies in flight land before the CTA exits (bounded)
    for (int64_t g = gstep - NS; g < gstep; ++g)
      if (g >= 0) mbar_wait_bounded(smem_u32(&full[g % NS]), (uint32_t)((g / NS) & 1), kStWaitLimit);
  } else {
    const int g = tid / tpr;  // 4-row group of this thread
    const int col = CW * (tid - g * tpr);
    const bool active = g < Gm::G;
    const int rx = g % Gm::RUNS, ly = g / Gm::RUNS;
    bool failed = false;
    for (int64_t item = blockIdx.x; item < items && !failed; item += gridDim.x) {
      const int tx = (int)(item % ntx);
      const int64_t r = item / ntx;
      const int ty = (int)(r % nty);
      const int pc = (int)(r / nty);
      const int x0t = tx * Gm::TX, y0t = ty * Gm::TY;
      const int pb = pc * pch, pe = min(n1, pb + pch);
      const int x0 = x0t + 4 * rx, y = DIM == 3 ? y0t + ly : 0;
      const bool rows = active && x0 < n1 && y < n1;
      VT aP[4], aC[4], aN[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) aP[i] = aC[i] = aN[i] = SV::zero();
      for (int p = pb - 1; p <= pe; ++p, ++gstep) {
        const int s = (int)(gstep % NS);
        const bool hasN = p + 1 >= pb && p + 1 < pe;
        const bool hasC = p >= pb && p < pe;
        const bool hasP = p - 1 >= pb && p - 1 < pe;
        const uint32_t ok = mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)((gstep / NS) & 1), kStWaitLimit);
        if (!ok || *(volatile int*)&abort_flag) {
          if (!ok) {
            atomicExch(err, 1);
            *(volatile int*)&abort_flag = 1;
          }
          failed = true;
          break;
        }
        const float* xs = xs_base + s * xs_floats;
        const float* vs = vs_base + (int64_t)s * Gm::VF;
        const float* bs = bs_base + s * bs_floats;
        // the update of plane p-1, complete once plane p's lines have been applied.  JACOBI
        // runs on the coefficients of the iteration matrix I - omega D^-1 A (slot T: omega /
        // a_qq), so y = aP + (omega / a_qq) b needs no copy of the old x.
        auto epilogue = [&]() {
          const int q = p - 1;
          const int64_t rbase = DIM == 3 ? ((int64_t)q * n1l + y) * n1l + x0 : (int64_t)q * n1l + x0;
          float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
          if (MODE == CSR_JACOBI) dv = lds4(vs + ((int64_t)T * Gm::TY + ly) * Gm::TX + 4 * rx);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (x0 + i >= n1) break;
            VT o = aP[i];
            if (WB) {
              const VT b = SV::ld(bs + ((int64_t)ly * Gm::TX + 4 * rx + i) * m + col);
              o = MODE == CSR_JACOBI ? SV::axpy(vcomp(dv, i), b, o) : SV::sub(b, o);
            }
            SV::st(Y + (rbase + i) * m + col, o);
          }
        };
        if (rows && p >= 0 && p < n1) {
#pragma unroll
          for (int dl = 0; dl < 3; ++dl) {  // lines y-1, y+1, then the centre line
            const int dy = dl == 0 ? -1 : (dl == 1 ? 1 : 0);
            if (DIM == 2 && dy != 0) continue;
            const int hl = DIM == 3 ? ly + 1 + dy : 0;  // staged line
            VT xl[6];
            const float* xrow = xs + ((int64_t)hl * (Gm::TX + 2) + 4 * rx) * m + col;
#pragma unroll
            for (int j = 0; j < 6; ++j) xl[j] = SV::ld(xrow + (int64_t)j * m);
            const int tl = DIM == 3 ? 3 * (dy + 1) : 0;
            const int tz = DIM == 3 ? 9 : 3;
#pragma unroll
            for (int role = 0; role < 3; ++role) {  // 0: plane p+1 (offset -1), 1: p, 2: p-1 (offset +1)
              if ((role == 0 && !hasN) || (role == 1 && !hasC) || (role == 2 && !hasP)) continue;
              VT(&acc)[4] = role == 0 ? aN : (role == 1 ? aC : aP);
#pragma unroll
              for (int dx = 0; dx < 3; ++dx) {
                const int t = tl + role * tz + dx;
                const float4 v = lds4(vs + ((int64_t)t * Gm::TY + ly) * Gm::TX + 4 * rx);
#pragma unroll
                for (int i = 0; i < 4; ++i) SV::fma(acc[i], vcomp(v, i), xl[i + dx]);
              }
            }
            if (dy == 0 && hasP) epilogue();  // last line: plane p-1 is complete
          }
        } else if (rows && hasP) {
          epilogue();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          aP[i] = aC[i];
          aC[i] = aN[i];
          aN[i] = SV::zero();
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
      }
    }
  }
  __syncthreads();
}

template <int DIM>
size_t st_stage_bytes(int m, bool with_b) {
  using Gm = StGeo<DIM>;
  return ((size_t)Gm::NL * (Gm::TX + 2) * m + Gm::VF + (with_b ? (size_t)Gm::TY * Gm::TX * m : 0)) * sizeof(float);
}

}  // namespace

// ------------------------------------------------------------------ setup
// Recognise the 3^d neighbour pattern of a square CSR level on an n1^d grid and upload
// the step-major coefficient layout.  Leaves A.st_val null when the level is not such a
// stencil (or too small to be worth it).
int stencil_setup(pase_ctx* h, const HostCSR& A, const std::vector<double>& dinv, DevCSR& d) {
  d.st_val = nullptr;
  d.st_dim = d.st_n1 = d.st_xp = 0;
  const int64_t N = A.nrows;
  if (N != A.ncols || N <= 0) return PASE_OK;
  for (int dim = 3; dim >= 2; --dim) {
    const int64_t n1 = (int64_t)llround(std::pow((double)N, 1.0 / dim));
    int64_t chk = 1;
    for (int k = 0; k < dim; ++k) chk *= n1;
    if (chk != N || n1 < 8 || n1 > (1 << 20)) continue;
    bool ok = true;
    for (int64_t i = 0; i < N && ok; ++i) {
      const int64_t xi = i % n1, yi = (i / n1) % n1, zi = dim == 3 ? i / (n1 * n1) : 0;
      for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
        const int64_t j = A.col[k];
        const int64_t xj = j % n1, yj = (j / n1) % n1, zj = dim == 3 ? j / (n1 * n1) : 0;
        if (std::llabs(xj - xi) > 1 || std::llabs(yj - yi) > 1 || std::llabs(zj - zi) > 1) {
          ok = false;
          break;
        }
      }
    }
    if (!ok) continue;
    const int T = dim == 3 ? 27 : 9, TX = dim == 3 ? 16 : 64, TY = dim == 3 ? 4 : 1;
    const int64_t VF = (int64_t)(T + 1) * TY * TX;
    const int64_t ntx = (n1 + TX - 1) / TX, nty = dim == 3 ? (n1 + TY - 1) / TY : 1;
    const int64_t steps = n1 + 2;
    std::vector<float> sv((size_t)(steps * nty * ntx * VF), 0.f);
    auto slot = [&](int64_t s, int64_t x, int64_t y, int t) -> size_t {
      const int64_t tx = x / TX, ty = dim == 3 ? y / TY : 0, lx = x % TX, lyy = dim == 3 ? y % TY : 0;
      return (size_t)(((((s * nty + ty) * ntx + tx) * (T + 1) + t) * TY + lyy) * TX + lx);
    };
    // the same layout for the damped-Jacobi iteration matrix I - omega D^-1 A (slot T:
    // omega / a_qq), so that a sweep is y = J x + (omega D^-1) b
    const double om = h->opt.omega;
    std::vector<float> sj(sv.size(), 0.f);
    for (int64_t i = 0; i < N; ++i) {
      const int64_t xi = i % n1, yi = (i / n1) % n1, zi = dim == 3 ? i / (n1 * n1) : 0;
      const int64_t qi = dim == 3 ? zi : yi;  // plane along the marching axis
      for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
        const int64_t j = A.col[k];
        const int64_t dx = j % n1 - xi, dy = (j / n1) % n1 - yi, dz = dim == 3 ? j / (n1 * n1) - zi : 0;
        const int64_t off = dim == 3 ? dz : dy;  // offset along the marching axis
        const int t = (int)((dx + 1) + 3 * (dy + 1) + (dim == 3 ? 9 * (dz + 1) : 0));
        sv[slot(qi + off + 1, xi, yi, t)] = (float)A.val[k];
        sj[slot(qi + off + 1, xi, yi, t)] = (float)((j == i ? 1.0 : 0.0) - om * dinv[i] * A.val[k]);
      }
      sv[slot(qi + 2, xi, yi, T)] = (float)dinv[i];
      sj[slot(qi + 2, xi, yi, T)] = (float)(om * dinv[i]);
    }
    PASE_TRY(dev_alloc_t(h, &d.st_val, sv.size()));
    PASE_CUDA(cudaMemcpy(d.st_val, sv.data(), sizeof(float) * sv.size(), cudaMemcpyHostToDevice));
    PASE_TRY(dev_alloc_t(h, &d.st_jval, sj.size()));
    PASE_CUDA(cudaMemcpy(d.st_jval, sj.data(), sizeof(float) * sj.size(), cudaMemcpyHostToDevice));
    d.st_omega = om;
    d.st_dim = dim;
    d.st_n1 = (int)n1;
    d.st_xp = 0;
    return PASE_OK;
  }
  return PASE_OK;
}

bool stencil_ok(const DevCSR& A, int mode, int m, int64_t ldx, int64_t ldy, double omega) {
  if (A.st_val == nullptr || !(mode == CSR_MV || mode == CSR_RESID || mode == CSR_JACOBI)) return false;
  if (mode == CSR_JACOBI && (A.st_jval == nullptr || omega != A.st_omega)) return false;  // J built for this omega
  if (m % 8 != 0 || m < 8 || m > 128 || (ldx > 0 && ldx != m) || (ldy > 0 && ldy != m)) return false;
  const size_t stage = A.st_dim == 3 ? st_stage_bytes<3>(m, true) : st_stage_bytes<2>(m, true);
  return 2 * stage <= 200 * 1024;
}

// ------------------------------------------------------------------ launch
int launch_stencil(pase_ctx* h, int mode, int m, const DevCSR& A, const float* X, const float* B, double omega,
                   float* Y) {
  // two columns per thread (twice the consumer warps at 64 registers) when chosen by the
  // autotuner and the threads fit in 512; else four
  const int cw = (A.st_cw == 2 && 16 * (m / 2) + 32 <= 512) ? 2 : 4;
  const int tpr = m / cw;
  const int dim = A.st_dim, n1 = A.st_n1;
  const int TX = dim == 3 ? 16 : 64, TY = dim == 3 ? 4 : 1;
  const int ntx = (n1 + TX - 1) / TX, nty = dim == 3 ? (n1 + TY - 1) / TY : 1;
  const int threads = (16 * tpr + 31) / 32 * 32 + 32;  // consumer warps + the producer warp
  const bool wb = mode == CSR_RESID || mode == CSR_JACOBI;
  const size_t stage = dim == 3 ? st_stage_bytes<3>(m, wb) : st_stage_bytes<2>(m, wb);
  // Resident consumer warps, not pipeline depth, set the rate (measured at 128^3, m = 56:
  // one CTA per SM 0.55 ms with 2 to 4 stages, two CTAs per SM 0.37 ms with 2), so two
  // CTAs per SM when their registers (128 per thread) and stages fit, each with as many
  // stages as shared memory leaves.
  int per_sm = (threads <= 256 || cw == 2) ? 2 : 1;
  if (A.st_per_sm == 1) per_sm = 1;
  int NS = (int)std::min<size_t>(kStMaxStages, (200 * 1024) / per_sm / stage);
  if (NS < 2) {
    per_sm = 1;
    NS = (int)std::min<size_t>(kStMaxStages, (200 * 1024) / stage);
  }
  const size_t smem = (size_t)NS * stage;
  // planes per work item: about st_items items per resident CTA (6 unless the autotuner
  // chose otherwise), at least 8 planes per item
  const int64_t tiles = (int64_t)ntx * nty;
  const int64_t want = (int64_t)h->num_sms * per_sm * std::max(1, A.st_items);
  int npc = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(1, n1 / 8), (want + tiles - 1) / tiles));
  const int pch = (n1 + npc - 1) / npc;
  npc = (n1 + pch - 1) / pch;
  const int64_t items = tiles * npc;
  const int grid = (int)std::min<int64_t>(items, (int64_t)h->num_sms * per_sm);
  auto s = h->stream;
  const float om = (float)omega;
  const float* coef = mode == CSR_JACOBI ? A.st_jval : A.st_val;
#define PASE_ST_GO(D, MD, CWV, MT, MB)                                                                        \
  do {                                                                                                        \
    PASE_TRY(ensure_max_smem((const void*)k_stencil<D, MD, CWV, MT, MB>, 200 * 1024));                        \
    k_stencil<D, MD, CWV, MT, MB><<<grid, threads, smem, s>>>(n1, m, tpr, ntx, nty, pch, npc, NS, coef, X, B, om, \
                                                               Y, h->tc_err);                                 \
  } while (0)
#define PASE_ST_LAUNCH(D, MD)                 \
  do {                                        \
    if (cw == 2) PASE_ST_GO(D, MD, 2, 512, 2); \
    else if (threads > 256)                   \
      PASE_ST_GO(D, MD, 4, 512, 1);           \
    else                                      \
      PASE_ST_GO(D, MD, 4, 256, 2);           \
  } while (0)
  if (dim == 3) {
    if (mode == CSR_JACOBI) PASE_ST_LAUNCH(3, CSR_JACOBI);
    else if (mode == CSR_RESID) PASE_ST_LAUNCH(3, CSR_RESID);
    else PASE_ST_LAUNCH(3, CSR_MV);
  } else {
    if (mode == CSR_JACOBI) PASE_ST_LAUNCH(2, CSR_JACOBI);
    else if (mode == CSR_RESID) PASE_ST_LAUNCH(2, CSR_RESID);
    else PASE_ST_LAUNCH(2, CSR_MV);
  }
#undef PASE_ST_LAUNCH
#undef PASE_ST_GO
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

}  // namespace pase
