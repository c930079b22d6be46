// Fifth-generation tensor-core primitives of sm_100+ (tcgen05 family, inline
// PTX) used by the TF32 colour pass: tensor-memory allocation, shared-memory
// matrix descriptors, the TF32 MMA with FP32 accumulation in tensor memory,
// its completion through an mbarrier, and tensor-memory loads.
//
// Operand layout: K-major without swizzle.  An operand tile of R rows and K
// columns (TF32, 4 bytes each) is stored as core matrices of 8 rows x 16
// bytes (8 x 4 elements, 128 contiguous bytes, row after row); element
// (r, k) lives at
//     (k % 4) * 4 + (r % 8) * 16 + (k / 4) * KSTRIDE + (r / 8) * RSTRIDE
// bytes from the tile start.  KSTRIDE (between core matrices along K) is the
// descriptor's leading byte offset and RSTRIDE (between groups of 8 rows) its
// stride byte offset.  One MMA instruction of kind::tf32 consumes K = 8 (two
// core matrices along K).
//
// Every wait here is bounded: a wait that runs out returns false and the
// caller records the failure and leaves (no device-side trap).
#pragma once

#include <stdint.h>

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (no swizzle, descriptor version 1 of
// sm_100, base offset 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t kstride, uint32_t rstride) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kstride >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((rstride >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32, both
// K-major, no negation, dense; N / 8 in bits 17..22, M / 16 in bits 24..28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Round an FP32 value to TF32 (round to nearest, ties away), kept in an FP32
// register: the tensor core then reads it exactly.
__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Tensor memory: one warp allocates `ncols` columns (power of two >= 32) and
// writes the base address to *slot; the same warp frees them at the end.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D (tensor memory) (+)= A (shared) x B (shared), issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1u : 0u)
      : "memory");
}

// Arrive once on the mbarrier when every MMA this thread issued so far has
// completed.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the completion of the mbarrier phase with the given parity, at
// most `tries` polls; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int tries = 1 << 20) {
  const uint32_t a = smem_u32(mbar);
  for (int it = 0; it < tries; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane (warp w
// reads lanes 32 (w % 4) .. 32 (w % 4) + 31; taddr carries the warp's lane
// base in bits 16..31 and the first column in bits 0..15).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  // the wait sits in the same statement, so no use of r[] can be scheduled
  // before the load has landed
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
