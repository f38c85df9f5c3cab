// Small helpers shared by the tcgen05 kernels (learned smoother, split-product GEMM):
// shared-memory addresses, UMMA shared-memory descriptors and a bounded mbarrier wait.
#pragma once
#include <cstdint>

namespace pase {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// UMMA shared-memory descriptor, K-major without swizzle: 8-row x 16-byte core matrices,
// lbo = byte distance between core matrices along K, sbo = along M (or N)
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;                // base offset 0, no swizzle
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 A and B (both K-major), FP32 D.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Poll an mbarrier phase at most `limit` times; 1 when the phase completed.
__device__ __forceinline__ uint32_t mbar_wait_bounded(uint32_t mbar_addr, uint32_t phase, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it)
    asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(done)
                 : "r"(mbar_addr), "r"(phase));
  return done;
}

}  // namespace pase
