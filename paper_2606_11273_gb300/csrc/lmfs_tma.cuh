// One-dimensional bulk asynchronous copies (TMA, cp.async.bulk) from global
// to shared memory that complete on an mbarrier, and a bounded wait on it.
#pragma once
#include <cstdint>

namespace lmfs {

static __device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// dst, src 16-byte aligned; bytes a multiple of 16.
static __device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
static __device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait on an mbarrier phase; returns false if the limit was reached.
static __device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// After the wait on tile `failed` of a two-buffer pipeline (tile t + 1 issued
// before tile t is waited on) ran out: wait, with the same bound, for the
// copies that may still be landing in shared memory (tiles `failed` and
// `failed` + 1), so that the block leaves none in flight when it returns.
static __device__ __forceinline__ void mbar_drain2(uint64_t* bars, int failed, int ntile) {
  for (int t = failed; t < ntile && t <= failed + 1; ++t) mbar_wait(&bars[t & 1], (uint32_t)((t >> 1) & 1));
}

}  // namespace lmfs
