// 5th-generation tensor cores (tcgen05) for the FP32 maxvol block product
// B = A P^{-1} (Section IV.B cross step).  Inline PTX for sm_103a: operands in
// shared memory in the canonical K-major layout without swizzle, the
// accumulator in tensor memory (TMEM), completion through an mbarrier.
//
// Canonical K-major layout of an R x K operand of 32-bit elements: "core
// matrices" of 8 rows x 16 bytes (4 elements) stored as 128 contiguous bytes;
// core matrices adjacent along K are 128 bytes apart (leading byte offset),
// 8-row groups are `sbo` bytes apart (stride byte offset).  One kind::tf32
// instruction consumes K = 8 (two core matrices along K).
#pragma once
#include <cstdint>

namespace ttp {
namespace tc {

constexpr int kRows = 128;  // MMA M: maxvol block rows (block_rows <= 128, padded with zeros)
constexpr uint32_t kWaitLimit = 1u << 24;  // bounded spin on the completion barrier
// The waits inside maxvol's visit loop may be shortened at build time (a test
// build makes them give up at once, to exercise the failure path); the wait
// before the accumulators are released keeps kWaitLimit, so no product is in
// flight when the tensor memory is freed.
#ifndef TTP_TC_LOOP_WAIT
#define TTP_TC_LOOP_WAIT (1u << 24)
#endif
constexpr uint32_t kLoopWaitLimit = TTP_TC_LOOP_WAIT;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) in a canonical K-major operand
__device__ __forceinline__ int kmaj(int row, int k, int sbo) {
  return (row >> 3) * sbo + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// padded K and N of a rank-rho block product: a multiple of 16 (N rule for M = 128)
__host__ __device__ __forceinline__ int pad16(int rho) { return (rho + 15) & ~15; }

// shared-memory matrix descriptor: start address, LBO = 128 B, SBO, version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::tf32: D F32, A and B TF32, both K-major, M = 128
__device__ __forceinline__ uint32_t instr_desc(int n, bool negate_b) {
  uint32_t i = (1u << 4) | (2u << 7) | (2u << 10);
  if (negate_b) i |= 1u << 14;
  i |= (uint32_t)(n >> 3) << 17;
  i |= (uint32_t)(kRows >> 4) << 24;
  return i;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(arrivals));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// wait for completion of phase `parity`; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit = kWaitLimit) {
  const uint32_t a = smem_u32(mbar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// whole warp: allocate `ncols` TMEM columns (power of two >= 32); the address lands in *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// whole warp: 8 consecutive 32-bit columns of the warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = __uint_as_float(r[c]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// TMEM columns for the accumulators D = Re A [Re M | Im M] and E = Im A [Re M | Im M]
// of a rank-r_max product
__host__ __device__ __forceinline__ uint32_t tmem_cols(int rmax) {
  const int need = 4 * pad16(rmax);
  uint32_t c = 32;
  while ((int)c < need) c <<= 1;
  return c;
}

}  // namespace tc
}  // namespace ttp
