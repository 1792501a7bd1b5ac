// sm_100-family primitives written as inline PTX: mbarriers, the async-proxy fence,
// and the fifth-generation tensor core (tcgen05: tensor-memory allocation, MMA from
// shared-memory descriptors, commit to an mbarrier, loads from tensor memory).
//
// Operand layout used with make_smem_desc (no swizzle, K-major): an operand of R rows
// and K 16-bit elements is stored as 8-row x 16-byte "core matrices" of 128 contiguous
// bytes; core matrix (row group m, K group kg) sits at byte offset
// (m * (K / 8) + kg) * 128, row r of it at + (r % 8) * 16, element k at + (k % 8) * 2.
// So the distance between core matrices adjacent in K (the leading-dimension offset)
// is 128 bytes and between row groups (the stride offset) K / 8 * 128 bytes; one MMA
// step of K = 16 covers two K groups, so step j starts at byte j * 256.
#pragma once
#include <cstdint>

namespace wcl {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ---- mbarriers ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes initialised barriers visible to the async proxy (tensor core, TMA)
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// polls until the phase with this parity has completed, at most `limit` times;
// false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long limit) {
  for (long k = 0; k < limit; k++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// orders this thread's generic-proxy shared-memory writes before later async-proxy
// reads (tensor copies, MMAs) of the same memory
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// ---- tensor memory -------------------------------------------------------------
// One warp (all lanes) allocates `ncols` columns (a power of two, at least 32) of
// tensor memory for the CTA; the TMEM address is written to shared memory at dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// ---- descriptors -----------------------------------------------------------------
// shared-memory matrix descriptor: start address, leading- and stride-dimension byte
// offsets (all in 16-byte units), descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t make_smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// instruction descriptor of kind::f16 with BF16 A and B (both K-major) and an FP32
// accumulator: D format bits 4-5 = 1 (F32), A format bits 7-9 = 1 (BF16), B format
// bits 10-12 = 1 (BF16), N / 8 at bits 17-22, M / 16 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// ---- MMA -------------------------------------------------------------------------
// D[tmem] (+)= A[smem] * B[smem]^T; accumulate = 0 overwrites D.  Issued by one thread.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// one arrive on the mbarrier once every MMA this thread issued before has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// ---- tensor memory -> registers ------------------------------------------------
// warp w may read lanes 32 (w % 4) .. 32 (w % 4) + 31; thread t gets lane base + t,
// eight consecutive 32-bit columns from the column in taddr
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int k = 0; k < 8; k++) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

}  // namespace wcl
