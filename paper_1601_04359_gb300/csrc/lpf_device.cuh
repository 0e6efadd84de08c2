// Device helpers shared by the library's kernels: bit-packed image staging,
// TMA bulk copies with bounded mbarrier waits, warp reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lpf {

// Bounded wait: spins at most this many try_wait rounds (each round may
// suspend the thread for a hardware-chosen time), then reports a timeout.
constexpr uint32_t kWaitRounds = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared, completion signalled on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Wait for phase `parity` of `bar`; false when the bounded wait (`rounds`
// try_wait rounds) gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t rounds = kWaitRounds) {
  for (uint32_t it = 0; it < rounds; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// The staged word a baked pixel word refers to.  A pixel word (and the first
// word of a pair) is (byte offset << 5) | funnel shift with a shift below 32,
// so the byte offset is a plain right shift by 5 (one add with a shifted
// operand, no masking), and the funnel shift reads the low 5 bits directly.
__device__ __forceinline__ const uint32_t* lane_word(const uint32_t* lane_base, uint32_t pix) {
  return reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(lane_base) + (pix >> 5));
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace lpf
