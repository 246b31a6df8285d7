// Inline-PTX helpers of the tcgen05 kernels: shared-memory addresses,
// cluster ranks and DSMEM addresses, mbarriers with bounded waits, and the
// shared-memory matrix descriptor of a K-major operand with 128-byte swizzle.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace hmm {
namespace tc {

constexpr long long TC_WAIT_CYCLES = 4000000000ll;   // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ uint64_t mbar_arrive(uint64_t* b) {
  uint64_t st;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(smem_u32(b)) : "memory");
  return st;
}
__device__ __forceinline__ uint64_t mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  uint64_t st;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(st)
               : "r"(smem_u32(b)), "r"(bytes)
               : "memory");
  return st;
}
// Bounded wait for the phase with the given parity; false once `limit` SM
// clock cycles have passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long long limit = TC_WAIT_CYCLES) {
  const uint32_t addr = smem_u32(b);
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}
// K-major operand with 128-byte swizzle: 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: FP16 A and B, FP32 D, both K-major.
constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Byte offset of element (row, k) in a [rows][64] FP16 K-block tile.
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  const int chunk = k >> 3;
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4) + ((k & 7) << 1));
}

}  // namespace tc
}  // namespace hmm

namespace hmm {
namespace tc {
// Instruction descriptor of kind::tf32: TF32 A and B (format 2), FP32 D,
// both K-major.
constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Byte offset of 16-byte chunk q (0..7) of row `row` in a [rows][128 B] tile
// with 128-byte swizzle (the layout sw128_desc describes).
__device__ __forceinline__ uint32_t sw128_chunk(int row, int q) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((q ^ (row & 7)) << 4));
}
}  // namespace tc
}  // namespace hmm
