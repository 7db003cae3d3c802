// Value-type operations used by the generic butterflies: badd(a, b) = a + b,
// bsub(a, b) = a - b.  Integers for host-side tests and the exact inverse;
// float and packed float2 (one f32x2 instruction per pair) on the device.
#pragma once

#ifdef __CUDACC__
#include <cuda_runtime.h>
#define ATDCT16_OPS_HD __host__ __device__ __forceinline__
#else
#define ATDCT16_OPS_HD inline
#endif

namespace atdct16 {

ATDCT16_OPS_HD int badd(int a, int b) { return a + b; }
ATDCT16_OPS_HD int bsub(int a, int b) { return a - b; }
ATDCT16_OPS_HD long long badd(long long a, long long b) { return a + b; }
ATDCT16_OPS_HD long long bsub(long long a, long long b) { return a - b; }

// Two exact int16 lanes in one 32-bit word, offset-binary: each 16-bit field
// holds value + 32768, so the word for lanes (lo, hi) is
// (lo + 32768) + 65536 (hi + 32768).  One 32-bit add of three operands adds
// or subtracts both lanes and re-biases them; no carry crosses lanes while
// every true lane value stays in [-32768, 32767].
struct Swar16 {
  unsigned v;
};
constexpr unsigned kSwarBias = 0x80008000u;
ATDCT16_OPS_HD Swar16 badd(Swar16 a, Swar16 b) { return Swar16{a.v + b.v - kSwarBias}; }
ATDCT16_OPS_HD Swar16 bsub(Swar16 a, Swar16 b) { return Swar16{a.v - b.v + kSwarBias}; }

// The same with the bias 4096: each field holds value + 4096, exact while
// every true lane value stays in [-4096, 61439].  A 1-D pass over 8-bit
// inputs never leaves [-4080, 4080] (at most 16 terms of magnitude <= 255),
// so its outputs are 13-bit field values that a byte permute can place
// directly into the mantissa of a float.
struct SwarRow {
  unsigned v;
};
constexpr unsigned kSwarRowBias = 0x10001000u;
ATDCT16_OPS_HD SwarRow badd(SwarRow a, SwarRow b) { return SwarRow{a.v + b.v - kSwarRowBias}; }
ATDCT16_OPS_HD SwarRow bsub(SwarRow a, SwarRow b) { return SwarRow{a.v - b.v + kSwarRowBias}; }

#ifdef __CUDACC__
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
  return (unsigned long long)__float_as_uint(v.x) | ((unsigned long long)__float_as_uint(v.y) << 32);
}
__device__ __forceinline__ float2 bits_f2(unsigned long long u) {
  return make_float2(__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32)));
}
__device__ __forceinline__ float2 badd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 bsub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(d);
}
__device__ __forceinline__ float badd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float bsub(float a, float b) { return __fsub_rn(a, b); }
#endif

// A value that may be known to be zero.  Where the flag is a compile-time
// fact (a butterfly unrolled over inputs that are zero by construction), the
// branches fold away: an addition with a zero operand costs nothing, and a
// subtraction from zero becomes one negation.  V needs badd, bsub and a
// value-initialised zero.
// (After every badd / bsub overload, so that the templates see them.)
template <class V>
struct MaybeZero {
  V v;
  bool z;
};
template <class V>
ATDCT16_OPS_HD MaybeZero<V> badd(MaybeZero<V> a, MaybeZero<V> b) {
  if (a.z) return b;
  if (b.z) return a;
  return MaybeZero<V>{badd(a.v, b.v), false};
}
template <class V>
ATDCT16_OPS_HD MaybeZero<V> bsub(MaybeZero<V> a, MaybeZero<V> b) {
  if (b.z) return a;
  if (a.z) return MaybeZero<V>{bsub(V{}, b.v), false};
  return MaybeZero<V>{bsub(a.v, b.v), false};
}

}  // namespace atdct16
