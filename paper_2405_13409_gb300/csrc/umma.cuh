// Fifth-generation tensor-core primitives (tcgen05) as inline PTX: tensor
// memory allocation, the single-thread BF16 MMA with an FP32 accumulator in
// tensor memory, its completion through an mbarrier (bounded waits), and
// loads of the accumulator into registers.
//
// Operands are K-major BF16 tiles in shared memory in the no-swizzle
// core-matrix layout: a core matrix is 8 rows x 16 bytes (8 BF16 along K)
// stored as 128 contiguous bytes; core matrices adjacent along K are 128
// bytes apart (the descriptor's leading byte offset) and 8-row groups are
// K x 16 bytes apart (its stride byte offset).  One MMA of kind::f16 takes
// K = 16, i.e. two core matrices along K, so step s of a K-loop starts 256 s
// bytes into the tile.
//
// For M = 128 and cta_group::1 the accumulator row i sits in tensor-memory
// lane i and column j in column base + j; warp w of the CTA may read lanes
// 32 (w % 4) .. 32 (w % 4) + 31 only.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace spoly {

// Byte offset of element (row, k) of a K-major BF16 tile with K columns.
SPOLY_HD constexpr int umma_off(int row, int k, int K) {
  return (row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0),
// N / 8 in bits 17-22, M / 16 in bits 24-28; dense, no negation.
constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

#ifndef SPOLY_HOST_BUILD
SPOLY_D uint32_t smem_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading
// byte offset / 16 (bits 16-29), stride byte offset / 16 (bits 32-45), the
// descriptor version of this architecture (bit 46 = 1), base offset 0, no
// swizzle (bits 61-63 = 0).
SPOLY_D uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// A whole warp allocates `cols` tensor-memory columns (a power of two, 32 to
// 512) and the base address lands in *slot; the CTA then gives up its right
// to allocate again, so that other CTAs on the SM are not held back.
SPOLY_D void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(slot)),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

// The allocating warp frees the columns before the CTA exits.
SPOLY_D void tmem_free(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols) : "memory");
}

// Order tensor-core operations around a thread barrier: `before` ahead of
// the barrier, `after` behind it in the thread that goes on to use tensor
// memory (issue an MMA, or read the accumulator).
SPOLY_D void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
SPOLY_D void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Makes this thread's ordinary shared-memory stores visible to the tensor
// core's operand reads (the async proxy); followed by a barrier.
SPOLY_D void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

SPOLY_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// One non-blocking poll (test_wait, unlike try_wait, returns at once): has
// the phase of the given parity completed?
SPOLY_D bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0u;
}

// Bounded wait for the phase of the given parity: false if it has not
// completed within `limit` SM clock cycles.
SPOLY_D bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// D (+)= A B for one K = 16 step, D in tensor memory at d_tmem, A (M x 16)
// and B (N x 16) K-major in shared memory; accumulate = 0 overwrites D.
// Issued by a single thread.
SPOLY_D void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The mbarrier receives one arrival when every tensor-core operation issued
// so far by this thread has completed.
SPOLY_D void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

// 32 consecutive FP32 accumulator columns of the warp's 32 lanes (thread i
// gets lane base + i), complete on return.
SPOLY_D void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
#endif

}  // namespace spoly
