// Thin wrappers over the sm_103a tensor-core and asynchronous-copy instructions used by
// the tensor-core kernels: tcgen05 (MMA with TMEM accumulators), mbarrier, 1-D bulk copies.
//
// Shared-memory operand descriptor (K-major): bits 0-13 start address >> 4, 16-29 leading
// byte offset >> 4 (no swizzle: distance between 8x16-byte core matrices along K), 32-45
// stride byte offset >> 4 (distance between 8-row groups along M or N), bits 46-48 = 0b001,
// 49-51 base offset, 61-63 swizzle mode (0 none, 2 128-byte).
// Instruction descriptor: bits 4-5 accumulator format (1 = F32), 7-9 / 10-12 A / B format
// (2 = TF32 for kind::tf32), 15 / 16 A / B major (0 = K-major), 17-22 N >> 3, 24-28 M >> 4.
// Every wait is bounded: it gives up after a fixed number of polls and reports failure.
#pragma once

#include <cstdint>

namespace fmmpc {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// K-major operand in the 128-byte swizzle: rows of 128 bytes (32 TF32 values of K), the
// 16-byte chunk c of row r stored at chunk position c ^ (r % 8).  The swizzle is applied to
// absolute shared-memory address bits, so with the base-offset field left at 0 the start may
// be any row of a 1024-byte-aligned buffer (and advanced by 32 bytes per K step of 8);
// sbo = 1024, the distance between 8-row groups.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                   // leading byte offset: unused in this mode
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// The same descriptor as two 32-bit words: the high word is the same for every operand of
// this layout, and the low word of an operand starting at saddr is its 16-byte address plus
// the leading-byte-offset field.  The address field cannot carry into bit 14 (shared memory
// is below 256 KB), so stepping a descriptor along K or along rows is an add to the low word:
// +2 per 32 bytes of K, +8 per 128-byte row.  Issue loops build descriptors this way because
// the MMA issuer is a single thread, and a few dependent 64-bit operations per MMA cost about
// as much as the MMA itself.
constexpr uint32_t SW128_HI = (1024u >> 4) | (1u << 14) | (2u << 29);
__device__ __forceinline__ uint32_t desc_lo(uint32_t saddr) { return ((saddr >> 4) & 0x3FFFu) | (1u << 16); }
__device__ __forceinline__ uint64_t desc_of(uint32_t lo) { return ((uint64_t)SW128_HI << 32) | lo; }

__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t M, uint32_t N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// kind::f16 (FP16 or BF16 operands as the instruction descriptor says, FP32 accumulation)
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar)));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }

// warp-wide
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 32 lanes x 16 consecutive 32-bit columns per thread (warp-wide), then wait
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count));
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes));
}

__device__ __forceinline__ bool mbar_test(uint64_t *mbar, uint32_t parity) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"(smem_addr(mbar)), "r"(parity));
  return r != 0;
}

// Suspends until the phase with the given parity completes or about hint_ns elapse.
__device__ __forceinline__ bool mbar_try(uint64_t *mbar, uint32_t parity, uint32_t hint_ns) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"(smem_addr(mbar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return r != 0;
}

// Waits for the barrier phase with the given parity; false after max_tries suspended
// tries of ~4 us (about a second) or when *abort becomes non-zero (another thread of the
// block gave up).  try_wait sleeps in hardware instead of spinning on shared memory, which
// would take bandwidth from the tensor core's operand reads.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, volatile int *abort,
                                          int max_tries = 1 << 18) {
  for (int i = 0; i < max_tries; ++i) {
    if (mbar_try(mbar, parity, 4000u)) return true;
    if (abort && *abort) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns per thread (warp-wide), then wait; the wait is
// in the same statement so no use of the registers can be scheduled before it
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 1-D bulk copy global -> shared, completion counted in bytes on mbar (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst_smem)),
               "l"(src_gmem), "r"(bytes), "r"(smem_addr(mbar))
               : "memory");
}

}  // namespace tc
}  // namespace fmmpc
