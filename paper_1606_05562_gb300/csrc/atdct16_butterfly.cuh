// 1-D 16-point butterflies of the multiplierless transform T of arXiv 1606.05562.
//
// Forward:  y = T x  with  T = P2 M4 M3 M2 P1 M1   (Sec. 2, factorisation Eq.)
// Inverse:  x = T^T y with T^T = M1 P1^T M2 M3^T M4 P2^T (M1, M2, M4 are
//           symmetric; M3^T transposes each printed 4x4 block).
//
// Each direction costs 16 + 16 + 24 + 4 = 60 additions (Table 1) and no
// multiplication.  The code is generic over the value type V: the caller
// provides  V badd(V, V)  and  V bsub(V, V)  for it (int on the host for unit
// tests, float / packed float2 on the device; see atdct16_ops.cuh).
//
// Reading of the printed permutation P2 (its cycle notation repeats the first
// element of two cycles): row i of T is row p(i) of M4 M3 M2 P1 M1 with
//   p = [0, 8, 4, 11, 3, 9, 5, 12, 1, 13, 7, 10, 2, 14, 6, 15].
#pragma once

#include "atdct16_ops.cuh"

#ifdef __CUDACC__
#define ATDCT16_HD __host__ __device__ __forceinline__
#else
#define ATDCT16_HD inline
#endif

namespace atdct16 {

// Forward 1-D transform y = T x (60 additions).
template <class V>
ATDCT16_HD void fwd16(const V (&x)[16], V (&y)[16]) {
  V a[16], c[16], d[16];
  // M1 = [[I8, J8], [J8, -I8]]
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    a[i] = badd(x[i], x[15 - i]);
    a[8 + i] = bsub(x[7 - i], x[8 + i]);
  }
  // P1 = diag(I9, printed 7x7 permutation): b[9 + r] = a[9 + q(r)],
  // q = [2, 3, 6, 5, 4, 1, 0].  Applied by renaming inside M2 below.
  const V b9 = a[11], b10 = a[12], b11 = a[15], b12 = a[14], b13 = a[13], b14 = a[10], b15 = a[9];
  const V b8 = a[8];
  // M2 = diag(B8, B8), B8 = [[I4, J4], [J4, -I4]]
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    c[i] = badd(a[i], a[7 - i]);
    c[4 + i] = bsub(a[3 - i], a[4 + i]);
  }
  c[8] = badd(b8, b15);
  c[9] = badd(b9, b14);
  c[10] = badd(b10, b13);
  c[11] = badd(b11, b12);
  c[12] = bsub(b11, b12);
  c[13] = bsub(b10, b13);
  c[14] = bsub(b9, b14);
  c[15] = bsub(b8, b15);
  // M3: four printed 4x4 blocks
  d[0] = badd(c[0], c[3]);
  d[1] = badd(c[1], c[2]);
  d[2] = bsub(c[2], c[1]);
  d[3] = bsub(c[0], c[3]);
  d[4] = badd(badd(c[5], c[6]), c[7]);            // [ 0  1  1  1]
  d[5] = bsub(c[7], badd(c[4], c[5]));            // [-1 -1  0  1]
  d[6] = bsub(c[5], badd(c[4], c[6]));            // [-1  1 -1  0]
  d[7] = badd(bsub(c[4], c[6]), c[7]);            // [ 1  0 -1  1]
  d[8] = badd(c[8], c[11]);
  d[9] = badd(c[9], c[10]);
  d[10] = bsub(c[10], c[9]);
  d[11] = bsub(c[11], c[8]);
  d[12] = badd(badd(c[13], c[14]), c[15]);        // [ 0  1  1  1]
  d[13] = bsub(badd(c[12], c[13]), c[15]);        // [ 1  1  0 -1]
  d[14] = badd(bsub(c[12], c[13]), c[14]);        // [ 1 -1  1  0]
  d[15] = badd(bsub(c[12], c[14]), c[15]);        // [ 1  0 -1  1]
  // M4 = diag(H2, I6, H2, I6) followed by P2
  y[0] = badd(d[0], d[1]);   // p(0) = 0
  y[8] = bsub(d[0], d[1]);   // p(8) = 1
  y[1] = badd(d[8], d[9]);   // p(1) = 8
  y[5] = bsub(d[8], d[9]);   // p(5) = 9
  y[12] = d[2];
  y[4] = d[3];
  y[2] = d[4];
  y[6] = d[5];
  y[14] = d[6];
  y[10] = d[7];
  y[11] = d[10];
  y[3] = d[11];
  y[7] = d[12];
  y[9] = d[13];
  y[13] = d[14];
  y[15] = d[15];
}

// Inverse 1-D transform x = T^T y (60 additions): the transposes of the
// forward stages, applied in reverse order.
template <class V>
ATDCT16_HD void inv16(const V (&y)[16], V (&x)[16]) {
  V c[16], a[16];
  // P2^T then M4 (symmetric): e[p(i)] = y[i]
  const V d0 = badd(y[0], y[8]);
  const V d1 = bsub(y[0], y[8]);
  const V d8 = badd(y[1], y[5]);
  const V d9 = bsub(y[1], y[5]);
  const V d2 = y[12], d3 = y[4], d4 = y[2], d5 = y[6], d6 = y[14], d7 = y[10];
  const V d10 = y[11], d11 = y[3], d12 = y[7], d13 = y[9], d14 = y[13], d15 = y[15];
  // M3^T (transposed 4x4 blocks)
  c[0] = badd(d0, d3);
  c[1] = bsub(d1, d2);
  c[2] = badd(d1, d2);
  c[3] = bsub(d0, d3);
  c[4] = bsub(d7, badd(d5, d6));                 // [ 0 -1 -1  1]
  c[5] = badd(bsub(d4, d5), d6);                 // [ 1 -1  1  0]
  c[6] = bsub(d4, badd(d6, d7));                 // [ 1  0 -1 -1]
  c[7] = badd(badd(d4, d5), d7);                 // [ 1  1  0  1]
  c[8] = bsub(d8, d11);
  c[9] = bsub(d9, d10);
  c[10] = badd(d9, d10);
  c[11] = badd(d8, d11);
  c[12] = badd(badd(d13, d14), d15);             // [ 0  1  1  1]
  c[13] = bsub(badd(d12, d13), d14);             // [ 1  1 -1  0]
  c[14] = bsub(badd(d12, d14), d15);             // [ 1  0  1 -1]
  c[15] = badd(bsub(d12, d13), d15);             // [ 1 -1  0  1]
  // M2 (symmetric)
  V b[16];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    b[i] = badd(c[i], c[7 - i]);
    b[4 + i] = bsub(c[3 - i], c[4 + i]);
    b[8 + i] = badd(c[8 + i], c[15 - i]);
    b[12 + i] = bsub(c[11 - i], c[12 + i]);
  }
  // P1^T: a[9 + q(r)] = b[9 + r]
#pragma unroll
  for (int i = 0; i < 9; ++i) a[i] = b[i];
  a[11] = b[9];
  a[12] = b[10];
  a[15] = b[11];
  a[14] = b[12];
  a[13] = b[13];
  a[10] = b[14];
  a[9] = b[15];
  // M1 (symmetric)
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    x[i] = badd(a[i], a[15 - i]);
    x[8 + i] = bsub(a[7 - i], a[8 + i]);
  }
}

// Number of non-zero entries in each row of T (the diagonal of T T^T, Sec. 2),
// read off the factorisation by running the butterfly on unit vectors
// (host code; the scaling S^2 = 1 / nnz and W = 48 / nnz follow from it).
inline void row_nonzeros(int nnz[16]) {
  for (int i = 0; i < 16; ++i) nnz[i] = 0;
  for (int j = 0; j < 16; ++j) {
    int x[16] = {0}, y[16];
    x[j] = 1;
    fwd16(x, y);
    for (int i = 0; i < 16; ++i) nnz[i] += (y[i] != 0);
  }
}

}  // namespace atdct16
