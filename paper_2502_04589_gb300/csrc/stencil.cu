// Structured-grid kernels of the FP32 smoothing path (damped-Jacobi sweep, residual,
// product) for operators that couple each node only to its 3^d grid neighbours.
//
// The step-(a) linear solve (Alg. 1 first step; Alg. 3 step 3) spends its time in damped
// Jacobi sweeps x <- x + omega D^-1 (b - A x) and residuals b - A x on the multigrid
// levels.  A Q1 operator on a uniform (n-1)^d interior grid with x-fastest ordering, and
// every Galerkin coarse operator of nested Q1 spaces, couples node (x, y, z) only to
// (x+dx, y+dy, z+dz) with |dx|, |dy|, |dz| <= 1, so its matrix needs no column indices.
// Setup recognises that pattern in a CSR level and stores the values by tap (a DIA
// layout): plane t = (dx+1) + 3(dy+1) + 9(dz+1) holds the coefficient of that neighbour
// for every row, plane 3^d holds 1 / a_ii, and the x extent of every plane is padded to a
// multiple of 4 (zeros) so that the coefficients of 4 consecutive x rows are one aligned
// 16-byte load.
//
// Why not the CSR kernel: with node-major multivectors [N][m] the CSR kernel gathers the
// m-wide X row of every nonzero, 27 times per row in 3D, and the L1 request rate, not
// HBM, bounds it.  Here a thread owns 4 consecutive x rows and one 16-byte column slice
// and marches through the grid along z (along y in 2D): each X value of plane p is loaded
// once per (dy, dx-window) and feeds the three output planes p-1, p, p+1 through three
// rolling register accumulators, so a thread issues 3 x 6 X loads per 4 x 3^3 row-taps
// instead of 108, and every operand stream (X, b, coefficients, y) is read or written
// once from HBM.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "pase_internal.h"

namespace pase {

namespace {

constexpr int kStRunX = 4;   // consecutive x rows per thread
constexpr int kStRuns3 = 4;  // x runs per tile row in 3D (tile x extent 16)

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void fma4(float4& a, float s, const float4& x) {
  a.x = fmaf(s, x.x, a.x);
  a.y = fmaf(s, x.y, a.y);
  a.z = fmaf(s, x.z, a.z);
  a.w = fmaf(s, x.w, a.w);
}
__device__ __forceinline__ float vcomp(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// acc[i] += sum_dx coef(t0 + dx + 1)[row i] * xl[i + dx + 1]  (i = 0..3)
__device__ __forceinline__ void tap_line(float4 (&acc)[kStRunX], const float4 (&xl)[kStRunX + 2],
                                         const float* __restrict__ vrow, int64_t P) {
#pragma unroll
  for (int dx = 0; dx < 3; ++dx) {
    const float4 v = ldg4(vrow + dx * P);
#pragma unroll
    for (int i = 0; i < kStRunX; ++i) fma4(acc[i], vcomp(v, i), xl[i + dx]);
  }
}

// MODE: CSR_MV (y = A x), CSR_RESID (y = b - A x), CSR_JACOBI (y = x + omega dinv (b - A x)).
// Work item = (tile, chunk of planes along the marching axis).  3D: tiles of 16 (x) by
// TY (y) nodes, a group of tpr threads per 4-row x run, march along z.  2D: tiles of
// 4 G x nodes, march along y.
template <int DIM, int MODE>
__global__ void __launch_bounds__(256, 2)
    k_stencil(int n1, int xp, int m, int tpr, int G, int TY, int ntx, int nty, int pch, int npc,
              const float* __restrict__ sv, int64_t P, const float* __restrict__ X, const float* __restrict__ B,
              float omega, float* __restrict__ Y) {
  constexpr int T = DIM == 3 ? 27 : 9;
  const int tid = threadIdx.x;
  const int g = tid / tpr;
  const int col = 4 * (tid - g * tpr);
  if (g >= G) return;
  const int64_t n1l = n1;
  const int64_t items = (int64_t)ntx * nty * npc;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int tx = (int)(item % ntx);
    const int64_t r = item / ntx;
    const int ty = (int)(r % nty);
    const int pc = (int)(r / nty);
    int x0, y;
    if (DIM == 3) {
      x0 = tx * (kStRuns3 * kStRunX) + (g % kStRuns3) * kStRunX;
      y = ty * TY + g / kStRuns3;
    } else {
      x0 = tx * (G * kStRunX) + g * kStRunX;
      y = 0;
    }
    if (x0 >= n1 || y >= n1) continue;
    const int pb = pc * pch, pe = min(n1, pb + pch);
    float4 aP[kStRunX], aC[kStRunX], aN[kStRunX];
#pragma unroll
    for (int i = 0; i < kStRunX; ++i) aP[i] = aC[i] = aN[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int p = pb - 1; p <= pe; ++p) {
      const bool hasN = p + 1 >= pb && p + 1 < pe;  // output plane p+1 (reads plane p with offset -1)
      const bool hasC = p >= pb && p < pe;
      const bool hasP = p - 1 >= pb && p - 1 < pe;
      if (p >= 0 && p < n1) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          if (DIM == 2 && dy != 0) continue;
          const int yy = y + dy;
          if (DIM == 3 && (unsigned)yy >= (unsigned)n1) continue;
          float4 xl[kStRunX + 2];
          const int64_t lbase = DIM == 3 ? ((int64_t)p * n1l + yy) * n1l : (int64_t)p * n1l;
#pragma unroll
          for (int j = 0; j < kStRunX + 2; ++j) {
            const int xx = x0 - 1 + j;
            xl[j] = (unsigned)xx < (unsigned)n1 ? ldg4(X + (lbase + xx) * m + col) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          // coefficient rows of the three output planes for this line's taps
          const int tl = DIM == 3 ? 3 * (dy + 1) : 0;      // (dy) part of the tap index
          const int tz = DIM == 3 ? 9 : 3;                  // stride of the marching offset
          const int64_t pstr = DIM == 3 ? n1l * xp : (int64_t)xp;
          const int64_t ybase = DIM == 3 ? (int64_t)y * xp + x0 : (int64_t)x0;
          if (hasN) tap_line(aN, xl, sv + (int64_t)(tl + 0 * tz) * P + (int64_t)(p + 1) * pstr + ybase, P);
          if (hasC) tap_line(aC, xl, sv + (int64_t)(tl + 1 * tz) * P + (int64_t)p * pstr + ybase, P);
          if (hasP) tap_line(aP, xl, sv + (int64_t)(tl + 2 * tz) * P + (int64_t)(p - 1) * pstr + ybase, P);
        }
      }
      if (hasP) {  // plane p-1 is complete
        const int q = p - 1;
        const int64_t rbase = DIM == 3 ? ((int64_t)q * n1l + y) * n1l + x0 : (int64_t)q * n1l + x0;
        float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MODE == CSR_JACOBI) {
          const int64_t pstr = DIM == 3 ? n1l * xp : (int64_t)xp;
          const int64_t ybase = DIM == 3 ? (int64_t)y * xp + x0 : (int64_t)x0;
          dv = ldg4(sv + (int64_t)T * P + (int64_t)q * pstr + ybase);
        }
#pragma unroll
        for (int i = 0; i < kStRunX; ++i) {
          if (x0 + i >= n1) break;
          const int64_t off = (rbase + i) * m + col;
          float4 o = aP[i];
          if (MODE == CSR_RESID || MODE == CSR_JACOBI) {
            const float4 b = ldg4(B + off);
            o = make_float4(b.x - o.x, b.y - o.y, b.z - o.z, b.w - o.w);
          }
          if (MODE == CSR_JACOBI) {
            const float4 xo = ldg4(X + off);
            const float d = omega * vcomp(dv, i);
            o = make_float4(fmaf(d, o.x, xo.x), fmaf(d, o.y, xo.y), fmaf(d, o.z, xo.z), fmaf(d, o.w, xo.w));
          }
          *reinterpret_cast<float4*>(Y + off) = o;
        }
      }
#pragma unroll
      for (int i = 0; i < kStRunX; ++i) {
        aP[i] = aC[i];
        aC[i] = aN[i];
        aN[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ setup
// Recognise the 3^d neighbour pattern of a square CSR level on an n1^d grid and upload
// the tap-plane layout (FP32 coefficients, then 1 / a_ii).  Leaves A.st_val null when the
// level is not such a stencil (or too small to be worth it).
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
    const int T = dim == 3 ? 27 : 9;
    const int64_t xp = (n1 + 3) / 4 * 4;
    const int64_t P = (dim == 3 ? n1 * n1 : n1) * xp;
    std::vector<float> sv((size_t)(T + 1) * P, 0.f);
    for (int64_t i = 0; i < N; ++i) {
      const int64_t xi = i % n1, yi = (i / n1) % n1, zi = dim == 3 ? i / (n1 * n1) : 0;
      const int64_t slot = (dim == 3 ? (zi * n1 + yi) : yi) * xp + xi;
      for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
        const int64_t j = A.col[k];
        const int64_t dx = j % n1 - xi, dy = (j / n1) % n1 - yi, dz = dim == 3 ? j / (n1 * n1) - zi : 0;
        const int t = (int)((dx + 1) + 3 * (dy + 1) + (dim == 3 ? 9 * (dz + 1) : 0));
        sv[(size_t)t * P + slot] = (float)A.val[k];
      }
      sv[(size_t)T * P + slot] = (float)dinv[i];
    }
    PASE_TRY(dev_alloc_t(h, &d.st_val, sv.size()));
    PASE_CUDA(cudaMemcpy(d.st_val, sv.data(), sizeof(float) * sv.size(), cudaMemcpyHostToDevice));
    d.st_dim = dim;
    d.st_n1 = (int)n1;
    d.st_xp = (int)xp;
    return PASE_OK;
  }
  return PASE_OK;
}

bool stencil_ok(const DevCSR& A, int mode, int m, int64_t ldx, int64_t ldy) {
  return A.st_val != nullptr && (mode == CSR_MV || mode == CSR_RESID || mode == CSR_JACOBI) && m % 8 == 0 &&
         m >= 8 && m <= 256 && (ldx <= 0 || ldx == m) && (ldy <= 0 || ldy == m);
}

// ------------------------------------------------------------------ launch
int launch_stencil(pase_ctx* h, int mode, int m, const DevCSR& A, const float* X, const float* B, double omega,
                   float* Y) {
  const int tpr = m / 4;
  int G = 16;
  while (G > 4 && G * tpr > 256) G /= 2;
  const int dim = A.st_dim, n1 = A.st_n1, xp = A.st_xp;
  const int64_t P = (int64_t)(dim == 3 ? n1 : 1) * n1 * xp;
  int TY = 1, ntx, nty;
  if (dim == 3) {
    TY = G / kStRuns3;
    ntx = (n1 + kStRuns3 * kStRunX - 1) / (kStRuns3 * kStRunX);
    nty = (n1 + TY - 1) / TY;
  } else {
    ntx = (n1 + G * kStRunX - 1) / (G * kStRunX);
    nty = 1;
  }
  // planes per work item: enough items for about four waves of two CTAs per SM
  const int64_t tiles = (int64_t)ntx * nty;
  const int64_t want = (int64_t)h->num_sms * 2 * 4;
  int npc = (int)std::max<int64_t>(1, std::min<int64_t>(n1, (want + tiles - 1) / tiles));
  const int pch = (n1 + npc - 1) / npc;
  npc = (n1 + pch - 1) / pch;
  const int64_t items = tiles * npc;
  const int threads = (G * tpr + 31) / 32 * 32;
  const int grid = (int)std::min<int64_t>(items, 0x7fffffff);
  auto s = h->stream;
  const float om = (float)omega;
#define PASE_ST_LAUNCH(D, MD)                                                                                   \
  k_stencil<D, MD><<<grid, threads, 0, s>>>(n1, xp, m, tpr, G, TY, ntx, nty, pch, npc, A.st_val, P, X, B, om, Y)
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
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}

}  // namespace pase
