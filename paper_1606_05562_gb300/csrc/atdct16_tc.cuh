// Fifth-generation tensor core (tcgen05) helpers for sm_103a: tensor-memory
// (TMEM) allocation, single-thread MMA issue with shared-memory matrix
// descriptors, completion through an mbarrier with bounded waits, TMEM ->
// register loads and the ordering fences between the threads' shared-memory
// writes, the tensor core's reads and the threads' TMEM reads.
//
// Operand layouts used here are the no-swizzle canonical ones, built from
// 8 x 16-byte "core matrices" (128 contiguous bytes).  For 16-bit elements,
// with LBO / SBO the descriptor's leading- and stride-dimension byte offsets:
//   K-major (rows of an M x K or N x K operand contiguous along K):
//     element (mn, k) at (mn & 7) * 16 + (k & 7) * 2 + (mn >> 3) * SBO + (k >> 3) * LBO
//   MN-major (columns contiguous along M or N):
//     element (mn, k) at (mn & 7) * 2 + (k & 7) * 16 + (mn >> 3) * SBO + (k >> 3) * LBO
// i.e. in both cases SBO steps between 8-wide groups along M (or N) and LBO
// between 8-deep groups along K (checked on GB300 with a one-CTA product of
// known operands: each order of the two offsets reproduces A B exactly only
// as stated).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace atdct16 {
namespace tc {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, LBO and SBO in
// 16-byte units, descriptor version 1 (bits 46-47), base offset 0.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with f16 A and B and an f32
// accumulator: D format (bits 4-5) = f32, A / B formats (bits 7-9, 10-12) =
// f16, A / B major (bits 15, 16: 0 K-major, 1 MN-major), N >> 3 (bits
// 17-22), M >> 4 (bits 24-28); dense, no negation, no saturation.
__host__ __device__ constexpr unsigned idesc_f16_f32(int m, int n, bool a_mn_major, bool b_mn_major) {
  return (1u << 4) | ((a_mn_major ? 1u : 0u) << 15) | ((b_mn_major ? 1u : 0u) << 16) |
         ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

// TMEM allocation of ncols columns (a power of two >= 32) by one whole warp;
// the TMEM address (lane 0, first column) is written to shared memory.
__device__ __forceinline__ void tmem_alloc(unsigned dst_smem, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[M x N] (TMEM, f32) = A B (+ D when accumulate); issued by one thread.
__device__ __forceinline__ void mma_f16(unsigned d_tmem, unsigned long long a_desc, unsigned long long b_desc,
                                        unsigned idesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1 : 0)
      : "memory");
}
// One arrival on the mbarrier once every MMA this thread issued so far has
// completed (its shared-memory reads included).
__device__ __forceinline__ void commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// The threads' generic-proxy shared-memory writes become visible to the
// tensor core's (async-proxy) reads.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive 32-bit columns of this thread's TMEM lane (shape 32x32b:
// warp w of the warpgroup reads lanes 32 (w & 3) .. + 31; taddr carries the
// warp's first lane in bits 16-31); ld_wait waits for it.
__device__ __forceinline__ void ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// mbarrier with an expected arrival count, its initialisation fence, and a
// bounded parity wait (false once about `cycles` SM clock cycles have
// passed; the SM cycle counter keeps running while the warp is suspended).
__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(unsigned mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity, long long cycles) {
  if (mbar_try_wait(mbar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 16; ++i)
      if (mbar_try_wait(mbar, parity)) return true;
    if (clock64() - t0 > cycles) return false;
  }
}

}  // namespace tc
}  // namespace atdct16
