// Device helpers shared by the fused kernels: packed-float and byte-packing
// value operations, the exact rounding of Z / 2304, the job search over a
// batch's descriptor table, the device status word, asynchronous copies and
// programmatic dependent launch.
#pragma once

#include <cuda_runtime.h>

#include "atdct16_internal.h"
#include "atdct16_ops.cuh"

namespace atdct16 {

// --------------------------------------------------------------------------
// Value types for the generic butterflies.
// --------------------------------------------------------------------------
__device__ __forceinline__ float2 f2mul(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }

__device__ __forceinline__ unsigned word_of(const uint4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// SwarRow word (fields f_lo, f_hi, each value + 4096 < 2^13) -> the exact
// floats 2^23 + 256 f = 2^23 + 2^20 + 256 value, one byte permute each.
__device__ __forceinline__ float2 swar_row_f2(unsigned w) {
  return make_float2(__uint_as_float(__byte_perm(w, 0x00004B00u, 0x5104u)),
                     __uint_as_float(__byte_perm(w, 0x00004B00u, 0x5324u)));
}

// Swar16 word (fields f_lo, f_hi < 2^16) -> the exact floats 2^23 + f, one
// byte permute each.
__device__ __forceinline__ float2 swar16_f2(unsigned w) {
  return make_float2(__uint_as_float(__byte_perm(w, 0x00004B00u, 0x5410u)),
                     __uint_as_float(__byte_perm(w, 0x00004B00u, 0x5432u)));
}

// d = (c << 16) | (sat_u8(a) << 8) | sat_u8(b)   (PTX cvt.pack semantics)
__device__ __forceinline__ unsigned pack_u8(unsigned a, unsigned b, unsigned c) {
  unsigned d;
  asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// d = (sat_s16(a) << 16) | sat_s16(b)
__device__ __forceinline__ unsigned pack_s16(int a, int b) {
  unsigned d;
  asm("cvt.pack.sat.s16.s32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Round half to even of x, clamped to 0..255, as the raw bits of a denormal:
// fl(x * 2^-149) lands on the denormal grid, whose spacing is 2^-149, so its
// bit pattern is rne(|x|) with the sign in bit 31.  As a signed 32-bit integer
// that saturates to 0 for negative x and to 255 above 255 in cvt.pack.sat.
__device__ __forceinline__ float2 rne_denormal(float2 x) {
  return __fmul2_rn(x, make_float2(__uint_as_float(1u), __uint_as_float(1u)));
}

// fp32(1/2304): with it, fl(Z * c) equals Z / 2304 exactly whenever Z / 2304 is
// a half-integer (Z is then a multiple of 9 and 9 * fp32(1/9) = 1 + 2^-27), and
// is within 6e-5 of Z / 2304 otherwise, far inside the 1/2304 gap to any .5.
static __constant__ float kInv2304 = 1.0f / 2304.0f;

// The job holding tile t: the last job with tile_begin <= t (tile_begin is
// increasing and jobs[0].tile_begin = 0), by binary search.
__device__ __forceinline__ void find_job(const ImageJob* __restrict__ jobs, int njobs, long long t, int& job) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&jobs[mid].tile_begin) <= t) lo = mid; else hi = mid - 1;
  }
  job = lo;
}

// The same job as a 32-way search by the whole warp:
// each round the lanes probe 32 evenly spaced jobs of the remaining range in
// parallel, so 512 jobs take two rounds of loads instead of nine dependent
// ones.  Every lane of the warp must call it; all get the same job.
__device__ __forceinline__ void warp_find_job(const ImageJob* __restrict__ jobs, int njobs,
                                              long long t, int& job) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = njobs;  // the job is in [lo, hi), jobs[lo].tile_begin <= t
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) >> 5;
    const int idx = lo + lane * step;
    const bool le = idx < hi && __ldg(&jobs[idx].tile_begin) <= t;
    const unsigned m = __ballot_sync(0xffffffffu, le);  // bit 0 is always set
    lo += (31 - __clz(m)) * step;
    hi = min(hi, lo + step);
  }
  job = lo;
}

__device__ __forceinline__ void set_status(int* status, int code) {
  atomicCAS(status, kDevOk, code);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct ZonalTile {
  const uint8_t* src;  // row 2j of block p of this lane
  uint8_t* dst;
  int src_pitch, dst_pitch;
  int nb;              // valid 16-pixel blocks in the tile (1..8)
  int t;               // tile index
  int r;
};

// Programmatic dependent launch: a kernel lets the next kernel of its stream
// (launched with the programmatic-serialisation attribute) be scheduled
// early; that kernel waits for this grid's completion and memory flush.  The
// fused kernels trigger as each CTA finishes its tiles, so the finalize's CTAs
// take the places of departing ones (a trigger at kernel start measured 2 us
// slower per call).
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_primary() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Exit of a fused kernel in a chain of programmatic dependent launches (one
// launch per class of zonal jobs): let the next kernel be scheduled, then wait
// until this kernel's predecessor has completed, so that this grid's
// completion implies its predecessor's and the last one's implies all of
// them (the PSNR finalize waits on the last).  Without a predecessor the wait
// returns at once.
__device__ __forceinline__ void pdl_chain_exit() {
  pdl_launch_dependents();
  pdl_wait_primary();
}

// Asynchronous 16-byte global -> shared copy (L2 only), its group commit and
// the wait until at most N of this thread's groups are still in flight.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
// The same with src_bytes (0 or 16) read and the rest of the 16 filled with zeros.
__device__ __forceinline__ void cp_async16_zfill(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gsrc), "r"(src_bytes) : "memory");
}
// An 8-byte copy (cached in L1 and L2: the 8-byte form has no L2-only variant)
// with src_bytes (0 or 8) read and the rest zero-filled.
__device__ __forceinline__ void cp_async8_zfill(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Host: launch with `smem` bytes of dynamic shared memory, as a programmatic
// dependent launch when `dependent` (the kernel may start before its
// predecessor on the stream has completed).
template <class... KArgs, class... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), int grid, int threads, int smem, cudaStream_t stream,
                           bool dependent, Args... args) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace atdct16
