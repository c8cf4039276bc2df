// Blackwell (sm_103a) tensor-core primitives: tcgen05 MMA with operands in
// shared memory and the accumulator in tensor memory (TMEM), mbarrier
// completion tracking with bounded waits, and the K-major no-swizzle operand
// layout.
//
// Operand layout (no swizzle): an operand is stored as "core matrices" of
// 8 x 16 bytes (8 strided 16-byte rows).  A buffer of R rows x C columns of
// bf16 written row by row puts element (r, c) at
//   (r/8) * (C/8) * 128 + (c/8) * 128 + (r%8) * 16 + (c%8) * 2.
// Read as a K-major operand (rows = M or N, columns = K) its descriptor has
// LBO = 128 (next 8 columns along K) and SBO = (C/8) * 128 (next 8 rows).
// Read as an MN-major operand (rows = K, columns = M or N; instruction
// descriptor transpose bit set) it has LBO = (C/8) * 128 (next 8 rows along
// K) and SBO = 128 (next 8 columns along M / N): in both cases LBO is the
// core-matrix stride along K and SBO the stride along M / N.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace nqs {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) of a K-major no-swizzle operand with K columns.
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, leading
// byte offset >> 4 in bits 16-29, stride byte offset >> 4 in bits 32-45,
// descriptor version 1 in bits 46-48, no base offset, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor for kind::f16 with BF16 A and B, FP32 accumulate,
// both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t make_idesc_bf16(int M, int N) {
  return (1u << 4)                      // D format: F32
       | (1u << 7)                      // A format: BF16
       | (1u << 10)                     // B format: BF16
       | ((uint32_t)(N >> 3) << 17)     // N / 8
       | ((uint32_t)(M >> 4) << 24);    // M / 16
}

// D[tmem] (+)= A[desc_a] * B[desc_b]^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t desc_a, uint64_t desc_b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem_d), "l"(desc_a), "l"(desc_b), "r"(idesc), "r"(accumulate));
}

// Arrive on the mbarrier once all previously issued MMAs of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               :
               : "r"(smem_addr(mbar)));
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Make this thread's generic-proxy shared-memory writes visible to the tensor core.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// TMEM allocation by one full warp; the address is written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
               :
               : "r"(smem_addr(slot)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" : : "r"(taddr), "r"(ncols));
}

// 16 consecutive 32-bit TMEM columns of this thread's lane (32x32b shape).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// mbarrier helpers.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" : : "r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Wait for the phase with the given parity to complete, giving up after
// max_iters polls.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_iters) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t it = 0; it < max_iters; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity));
    if (done) return true;
  }
  return false;
}

// Bound, in polls of mbarrier.try_wait, of the waits that may give up (and
// record NQS_ETIMEOUT).  Every translation unit that includes this header has
// its own copy; the host sets all of them through nqs_set_wait_limit, which
// exists to exercise the give-up path.  The drain below always uses the
// default bound, so TMEM is never freed under a running MMA.
constexpr uint32_t kDefaultWaitPolls = 1u << 26;
static __device__ uint32_t g_wait_polls = kDefaultWaitPolls;

// Drain before TMEM is freed.  After a bounded wait gave up, MMAs committed
// earlier (some never waited for) may still be running and writing TMEM.
// Every MMA-issuing thread of the CTA calls this once: it commits once more to
// `drain` (initialised with one arrival per issuing thread), whose phase 0
// completes when every MMA those threads issued has completed, and waits for
// it with the same bound.
__device__ __forceinline__ void drain_mmas(uint64_t* drain, uint32_t max_iters) {
  mma_commit(drain);
  mbar_wait(drain, 0, max_iters);
}

// Barrier over `count` threads with id `id` (1..15), OR-reducing a predicate.
__device__ __forceinline__ bool group_barrier_or(bool v, uint32_t id, uint32_t count) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.cta.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void group_barrier(uint32_t id, uint32_t count) {
  asm volatile("barrier.cta.sync %0, %1;\n" : : "r"(id), "r"(count) : "memory");
}
// Arrive on barrier `id` without waiting (the producer side of a hand-off).
__device__ __forceinline__ void group_arrive(uint32_t id, uint32_t count) {
  asm volatile("barrier.cta.arrive %0, %1;\n" : : "r"(id), "r"(count) : "memory");
}

}  // namespace tc
}  // namespace nqs
