// Zig-zag scan of a 16x16 block (Sec. 4: the image-compression procedure
// keeps the first r coefficients of this scan; the paper adapts the 8x8 JPEG
// scan to 16x16): anti-diagonals s = u + v in increasing order, even s walked
// with u decreasing, odd s with v decreasing (u = vertical frequency).  The
// same order is the block layout of the zig-zag coefficient and level option.
#pragma once

#ifdef __CUDACC__
#define ATDCT16_ZZ_HD __host__ __device__ __forceinline__
#else
#define ATDCT16_ZZ_HD inline
#endif

namespace atdct16 {

// (16 u + v) of the coefficient at scan position k, 0 <= k < 256.
ATDCT16_ZZ_HD int zigzag_word(int k) {
  int s = 0, base = 0;
  while (s < 30) {
    const int len = s < 16 ? s + 1 : 31 - s;
    if (k < base + len) break;
    base += len;
    ++s;
  }
  const int off = k - base, hi = s < 16 ? s : 15;
  const int a = hi - off, b = s - a;  // even s: u = a (decreasing); odd s: v = a (decreasing)
  return (s & 1) ? 16 * b + a : 16 * a + b;
}

// Scan position of the coefficient (u, v) = (word >> 4, word & 15): the
// inverse of zigzag_word.  Diagonal s = u + v starts after s (s + 1) / 2
// positions (s <= 15) or 256 - (31 - s)(32 - s) / 2 (s >= 16); along it the
// offset counts down from min(s, 15) in u (even s) or in v (odd s).
ATDCT16_ZZ_HD int zigzag_rank(int word) {
  const int u = word >> 4, v = word & 15, s = u + v;
  const int base = s <= 15 ? s * (s + 1) / 2 : 256 - (31 - s) * (32 - s) / 2;
  const int hi = s < 16 ? s : 15;
  return base + hi - ((s & 1) ? v : u);
}

}  // namespace atdct16
