// pase_residual_noalloc: the block residual of pase_residual for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running under a memory pool or arena that
// owns every device byte (a serving process that reserves the GPU up front), plugins
// hosted by another runtime that forbids allocation inside its callbacks, and code paths
// that must not allocate for latency or determinism reasons.  This entry point takes
// every input and output from the caller and keeps its only scratch (per-block partial
// sums of the column norms) in a fixed file-scope device array, so it performs no device
// allocation at all.
#include <mutex>

#include "pase_internal.h"

namespace pase {

// Largest block width accepted, and the number of partial-sum rows: one per block of the
// residual kernel, whose grid launch_csr caps at kReduceBlocksHost (the same constant, so
// the partial sums of any launch fit).
constexpr int kNoAllocMaxM = 64;
constexpr int kNoAllocBlocks = kReduceBlocksHost;
constexpr size_t kNoAllocScratchDoubles = (size_t)kNoAllocBlocks * 2 * kNoAllocMaxM + 2 * kNoAllocMaxM;

// The scratch lives for the lifetime of the process on every device that loads the
// library: 1216 x 128 + 128 doubles = 1.19 MiB.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code only holds a
// host-side stand-in under the array's name, so the address is looked up once per device
// (with that device current) and cached.
int scratch_address(double** out) {
  int dev = 0;
  PASE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PASE_ERR_INVALID_ARG, "pase_residual_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(PASE_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return PASE_OK;
}

// Device memory of the current device (managed memory counts): a pointer into another
// GPU's memory would be dereferenced without peer access by kernels launched here.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}
}  // namespace
}  // namespace pase

using namespace pase;

extern "C" int pase_residual_noalloc(int64_t n, int m, const int64_t* rowptr, const int32_t* colind,
                                     const double* A_val, const double* M_val, const double* U,
                                     const double* lambda, double* R, double* relres, void* cuda_stream) {
  if (n < 0 || m <= 0 || m % 8 != 0)
    return fail(PASE_ERR_INVALID_ARG, "pase_residual_noalloc: m must be a positive multiple of 8");
  if (m > kNoAllocMaxM)
    return fail(PASE_ERR_INVALID_ARG, "pase_residual_noalloc: m exceeds the fixed scratch (at most 64 columns)");
  if (n > INT32_MAX) return fail(PASE_ERR_INVALID_ARG, "pase_residual_noalloc: too many rows");
  if (!rowptr || !colind || !A_val || !M_val || !U || !lambda || !relres)
    return fail(PASE_ERR_INVALID_ARG, "pase_residual_noalloc: null argument");
  int dev = 0;
  PASE_CUDA(cudaGetDevice(&dev));
  const void* ptrs[] = {rowptr, colind, A_val, M_val, U, lambda, relres};
  for (const void* p : ptrs)
    if (!on_device(p, dev))
      return fail(PASE_ERR_INVALID_ARG, "pase_residual_noalloc: every array must be device memory of the current device");
  if (R && !on_device(R, dev))
    return fail(PASE_ERR_INVALID_ARG, "pase_residual_noalloc: R must be device memory of the current device");
  if (((uintptr_t)U | (uintptr_t)(R ? R : U)) % 16 != 0)
    return fail(PASE_ERR_INVALID_ARG, "pase_residual_noalloc: U and R must be 16-byte aligned");
  double* scratch = nullptr;
  PASE_TRY(scratch_address(&scratch));
  // A context on the stack carries the stream into the launchers; it owns no memory.
  pase_ctx ctx;
  ctx.stream = (cudaStream_t)cuda_stream;
  DevCSR A;
  A.nrows = n;
  A.ncols = n;
  A.rowptr = const_cast<int64_t*>(rowptr);
  A.col = const_cast<int32_t*>(colind);
  A.val = const_cast<double*>(A_val);
  double* partial = scratch;
  double* norms = scratch + (size_t)kNoAllocBlocks * 2 * kNoAllocMaxM;
  if (n == 0) {  // empty block: zero norms (relative residuals come out infinite)
    PASE_TRY(launch_fill(&ctx, 2 * m, 0.0, norms));
    return launch_relres(&ctx, m, norms, lambda, relres);
  }
  int nb = 0;
  // every block writes all 2m of its partial sums and the reduction reads exactly those,
  // so nothing in the scratch needs clearing between calls; nb <= kNoAllocBlocks by the
  // grid cap of launch_csr
  PASE_TRY(launch_csr<double>(&ctx, CSR_EIGRES, m, A, A_val, M_val, U, nullptr, nullptr, nullptr, lambda, 0.0,
                              R, nullptr, partial, &nb));
  PASE_TRY(launch_reduce_partials(&ctx, nb, 2 * m, partial, norms));
  PASE_TRY(launch_relres(&ctx, m, norms, lambda, relres));
  return PASE_OK;
}
