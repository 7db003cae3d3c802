// Fused zonal compression for small zonal extents (the Sec. 4 procedure with
// the r lowest zig-zag coefficients kept), and the host logic that splits a
// batch of zonal jobs into classes by the extent of their kept set.
//
// Why a separate kernel.  For r <= 36 every kept coefficient (u, v) has
// u + v <= 7, so it lies in the K x K low-frequency corner of the block with
// K = 1 (r = 1), 3 (r <= 6), 6 (r <= 21) or 8 (r <= 36).  Then
//   * the forward transform is needed only for the K lowest frequencies: the
//     row pass computes K of its 16 outputs and the column pass runs on K
//     columns and computes K outputs (46 of the 60 additions of Sec. 2 for
//     K = 8, fewer for smaller K; the unused outputs are dead code);
//   * the inverse has only K non-zero inputs in each direction (38 of 60
//     additions for K = 8, none at all for K = 1: there the kernel sums
//     each block with dp4a and stores the rounded constant 9 Y[0][0] / 2304);
//   * the squared error needs no dropped coefficient: with the orthonormal
//     C_hat, SSE = ||X - X_hat||^2 = ||X||^2 - ||B'||^2, and both terms are
//     exact integers here.  With pixels centred at 128 (which changes only
//     Y[0][0] and leaves the error unchanged) each block gives
//       2304 SSE = 2304 sum (x - 128)^2 - sum_kept W_u W_v Y_c[u][v]^2,
//     Y_c the coefficients of the centred block, W = 48 S^2 = 48 / nnz
//     (Sec. 2).  The pixel term comes from dp4a over the input bytes, the
//     coefficient term from exact 32-bit squares (|Y_c| <= 32768)
//     accumulated in 64 bits.
//
// Work decomposition (one warp per 16 x 128 tile of eight blocks, as in the
// general kernel): lane (p, j) = (lane & 3, lane >> 2) holds blocks p and
// p + 4 side by side in int16 SWAR words (Swar16: two offset-binary fields
// per 32-bit word, one 3-operand add per butterfly addition).
//   row pass      rows 2j, 2j+1: outputs c < K, the DC output centred by
//                 -2048 (pixels centred at 128);
//   transpose     t1 (words): word p 168 + c 20 + row;
//   column pass   column c = j: outputs u < K (exact int16 fields);
//   scale         D = keep W_u W_c Y_c per kept coefficient as one exact FMA
//                 on the float 2^23 + field; the DC coefficient of column 0
//                 also takes 2304 * 128 back, which adds 128 to every pixel
//                 of the reconstruction and undoes the centring;
//   inverse col.  on f32x2 (blocks p, p + 4), K non-zero inputs, into
//   transpose     t2 (float2): unit p 148 + c 18 + row;
//   inverse row   rows 2j, 2j+1: the integer numerator Z of X_hat = Z / 2304
//                 (every node below 2^24: exact), round half to even,
//                 clamp, store u8 (the general kernel's exact rounding).
// Both transposes are conflict-free (checked per quarter-/half-warp for the
// 16- and 8-byte accesses).  Blocks past the image edge are zero-filled by
// the input copies; a zero block reconstructs exactly (its DC is kept), so
// it contributes exactly 0 to the tile's squared error.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "atdct16_butterfly.cuh"
#include "atdct16_device.cuh"
#include "atdct16_internal.h"
#include "atdct16_zigzag.cuh"

namespace atdct16 {

// Packed float pairs (blocks p and p + 4) that may be known to be zero: the
// inputs of the inverse at or above K.
using ZF2 = MaybeZero<float2>;

constexpr int kBoxT1Words = 168;  // forward transpose: words per block pair (8 columns x 20, padded)
constexpr int kBoxT2Units = 148;  // back-transpose: float2 units per block pair (8 columns x 18, padded)
constexpr int kBoxFixedBytes = 4 * 4 * kBoxT1Words + 8 * 4 * kBoxT2Units;  // both transposes, 7424 bytes
constexpr int kBoxSlotBytes = 4 * 32 * 16;  // one staging slot: a tile's input rows, 4 x 16 bytes per lane
__host__ __device__ constexpr int box_warp_smem(int depth) { return kBoxFixedBytes + depth * kBoxSlotBytes; }

// Largest r whose kept zig-zag prefix lies in the K x K corner: the scan
// walks the anti-diagonals s = u + v in order, so the prefix stays inside
// while it covers only s < K, i.e. its first K (K + 1) / 2 coefficients.
__host__ __device__ constexpr int box_max_r(int k) { return k * (k + 1) / 2; }

// rne(z / 2304) of one exact integer z as raw denormal bits: the products of
// rne_denormal(f2mul(., kInv2304)) for one lane.
__device__ __forceinline__ unsigned round_dc(float z) {
  return __float_as_uint(__fmul_rn(__fmul_rn(z, kInv2304), __uint_as_float(1u)));
}

struct BoxTile {
  const uint8_t* src;  // row 2j of block p of this lane
  uint8_t* dst;
  int src_pitch, dst_pitch;
  int nb;              // valid 16-pixel blocks in the tile (1..8)
  int t;               // index of the tile's partial in the caller's numbering
  int r;
};

// Launch shape (chosen by the batch autotuner): K the extent, D the staging
// depth (tiles whose input rows are in flight, D slots per warp), the warps
// per CTA (tiles per CTA, from the block size) and the width in bytes of the
// input copies (vec: 16, one block row per copy, or 8).
template <int K, int D>
__global__ void __launch_bounds__(256, 2)
zonal_box_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles_ll,
                 const float2* __restrict__ wtab, float* __restrict__ tile_sse, int* __restrict__ status,
                 int pdl_early, int vec) {
  static_assert(K >= 1 && K <= 8 && D >= 1 && D <= 3, "box extent and staging depth");
  extern __shared__ __align__(16) unsigned char bsmem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, cta_warps = blockDim.x >> 5;
  const int p = lane & 3, j = lane >> 2;
  unsigned char* const wbase = bsmem + warp * box_warp_smem(D);
  unsigned* const t1 = reinterpret_cast<unsigned*>(wbase);
  float2* const t2 = reinterpret_cast<float2*>(wbase + 4 * 4 * kBoxT1Words);
  uint4* const stg = reinterpret_cast<uint4*>(wbase + kBoxFixedBytes) + lane;  // slot s: + 128 s
  const int ntiles = (int)ntiles_ll;  // the launcher checks ntiles < 2^30

  const int nwarps = gridDim.x * cta_warps;
  const int per_warp = (ntiles + nwarps - 1) / nwarps;
  const int t_first = (blockIdx.x * cta_warps + warp) * per_warp;
  const int t_stop = min(ntiles, t_first + per_warp);
  if (pdl_early) pdl_launch_dependents();  // the next class's kernel may be scheduled
  if (t_first >= t_stop) {
    pdl_chain_exit();
    return;
  }

  // ---- the warp's tile cursor (as in the general kernel)
  int c_t = 0, c_end = 0, tiles_x = 1, tx = 0, nb_last = 8, r_job = 0, src_pitch = 0, dst_pitch = 0, t_shift = 0;
  const uint8_t* src_band = nullptr;
  uint8_t* dst_band = nullptr;
  auto enter = [&](int t) -> bool {
    int job;
    warp_find_job(jobs, njobs, t, job);
    const ImageJob* J = jobs + job;
    const long long tb = __ldg(&J->tile_begin);
    tiles_x = __ldg(&J->tiles_x);
    const long long te = tb + (long long)tiles_x * (__ldg(&J->height) >> 4);
    if (t < tb || t >= te || tiles_x < 1) return false;
    c_end = (int)min(te, (long long)t_stop);
    const int lt = (int)(t - tb);
    const int ty = lt / tiles_x;
    tx = lt - ty * tiles_x;
    t_shift = (int)(__ldg(&J->level_base) - tb);
    src_pitch = (int)__ldg(&J->src_pitch);
    dst_pitch = (int)__ldg(&J->dst_pitch);
    const long long row = (long long)ty * kTileH + 2 * j;
    src_band = reinterpret_cast<const uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->src))) +
               row * src_pitch + 16 * p;
    dst_band = reinterpret_cast<uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->dst))) +
               row * dst_pitch + 16 * p;
    nb_last = min(8, (__ldg(&J->width) - (tiles_x - 1) * kTileW) >> 4);
    r_job = __ldg(&J->param);
    c_t = t;
    return true;
  };
  auto take = [&](BoxTile& z) {
    z.src = src_band + tx * kTileW;
    z.dst = dst_band + tx * kTileW;
    z.src_pitch = src_pitch;
    z.dst_pitch = dst_pitch;
    z.nb = tx == tiles_x - 1 ? nb_last : 8;
    z.t = c_t + t_shift;
    z.r = r_job;
  };
  auto advance = [&]() -> bool {
    ++c_t;
    if (++tx == tiles_x) {
      tx = 0;
      src_band += (long long)kTileH * src_pitch;
      dst_band += (long long)kTileH * dst_pitch;
    }
    return c_t >= t_stop || c_t < c_end || enter(c_t);
  };
  // Rows 2j, 2j+1 of blocks p, p + 4 into staging slot st (word k = row
  // 2j + (k & 1) of block p + 4 (k >> 1)); blocks past the image edge are
  // zero-filled without reading (the address stays inside the tile's row).
  auto issue = [&](const BoxTile& z, int st) {
    uint4* const d = stg + 128 * st;
    const int na = p < z.nb ? 16 : 0, nb4 = p + 4 < z.nb ? 16 : 0;
    const uint8_t* sa = na ? z.src : z.src - 16 * p;
    const uint8_t* sb = nb4 ? z.src + 64 : sa;
    if (vec == 16) {
      cp_async16_zfill(d, sa, na);
      cp_async16_zfill(d + 32, sa + (na ? z.src_pitch : 0), na);
      cp_async16_zfill(d + 64, sb, nb4);
      cp_async16_zfill(d + 96, sb + (nb4 ? z.src_pitch : 0), nb4);
    } else {  // two 8-byte copies per block row
      unsigned char* const d8 = reinterpret_cast<unsigned char*>(d);
      cp_async8_zfill(d8, sa, na >> 1);
      cp_async8_zfill(d8 + 8, sa + (na ? 8 : 0), na >> 1);
      cp_async8_zfill(d8 + 512, sa + (na ? z.src_pitch : 0), na >> 1);
      cp_async8_zfill(d8 + 520, sa + (na ? z.src_pitch + 8 : 0), na >> 1);
      cp_async8_zfill(d8 + 1024, sb, nb4 >> 1);
      cp_async8_zfill(d8 + 1032, sb + (nb4 ? 8 : 0), nb4 >> 1);
      cp_async8_zfill(d8 + 1536, sb + (nb4 ? z.src_pitch : 0), nb4 >> 1);
      cp_async8_zfill(d8 + 1544, sb + (nb4 ? z.src_pitch + 8 : 0), nb4 >> 1);
    }
    cp_async_commit();
  };

  if (!enter(t_first)) {
    if (lane == 0) set_status(status, kDevBadJob);
    pdl_chain_exit();
    return;
  }
  bool ok = true;
  // scale of this lane's column c = j for the warp's current r: integer
  // weights keep W_u W_c and the FMA constants that turn the float
  // 2^23 + field (field = Y_c + 32768) into keep W_u W_c Y_c
  int wr = -1;
  unsigned kwi[K];
  float kwf[K];
#pragma unroll
  for (int u = 0; u < K; ++u) kwi[u] = 0u, kwf[u] = 0.f;

  auto row_pass = [&](const uint4 (&X)[4], Swar16 (&rv)[2][16]) {
#pragma unroll
    for (int tr = 0; tr < 2; ++tr) {
      const uint4& wa = X[tr];
      const uint4& wb = X[2 + tr];
      Swar16 xs[16];
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const unsigned lo = __byte_perm(word_of(wa, w), word_of(wb, w), 0x5410u);  // a0 a1 b0 b1
        const unsigned hi = __byte_perm(word_of(wa, w), word_of(wb, w), 0x7632u);  // a2 a3 b2 b3
        xs[4 * w + 0].v = (lo & 0x00FF00FFu) | kSwarBias;
        xs[4 * w + 1].v = __byte_perm(lo, kSwarBias, 0x7351u);
        xs[4 * w + 2].v = (hi & 0x00FF00FFu) | kSwarBias;
        xs[4 * w + 3].v = __byte_perm(hi, kSwarBias, 0x7351u);
      }
      fwd16(xs, rv[tr]);  // only the outputs c < K are used
      rv[tr][0].v -= 0x08000800u;  // pixels centred at 128
    }
  };
  auto pixel_energy = [&](const uint4 (&X)[4]) -> unsigned {
    unsigned e = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      e = __dp4a(X[k].x, X[k].x, e);
      e = __dp4a(X[k].y, X[k].y, e);
      e = __dp4a(X[k].z, X[k].z, e);
      e = __dp4a(X[k].w, X[k].w, e);
    }
    return e;
  };

  // the warp's next D tiles: q[0] is the current one, its input rows in slot
  // st; q[i] in slot (st + i) mod D
  BoxTile q[D];
  bool hq[D];
  take(q[0]);
  ok = advance();
  issue(q[0], 0);
  hq[0] = true;
#pragma unroll
  for (int i = 1; i < D; ++i) {
    hq[i] = hq[i - 1] && ok && c_t < t_stop;
    if (hq[i]) {
      take(q[i]);
      ok = advance();
      issue(q[i], i);
    } else {
      cp_async_commit();
    }
  }
  int st = 0;
  while (true) {
    BoxTile& cur = q[0];
    cp_async_wait<D - 1>();  // the current tile's copies (the oldest group in flight)
    uint4 X[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) X[k] = stg[128 * st + 32 * k];
    if (cur.r != wr) {  // warp-uniform
      if (cur.r < 1 || cur.r > box_max_r(K)) {  // a job of another class: leave its tiles alone
        if (lane == 0) set_status(status, kDevBadJob);
        ok = false;
        break;
      }
      const float2* wt = wtab + (long long)cur.r * 256 + j * 16;  // [r][c][u], (keep, 1 - keep) W_u W_c / 256
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const float w = 256.0f * __ldg(&wt[u]).x;  // exact small integer
        kwf[u] = w;
        kwi[u] = (unsigned)__float2uint_rn(w);
      }
      wr = cur.r;
    }
    const bool va = p < cur.nb, vb = p + 4 < cur.nb;

    const unsigned ex = pixel_energy(X);  // dp4a over the 64 input bytes
    unsigned long long ke = 0ull;
    long long dc_term = 0;
    BoxTile fut;
    bool have_fut;
    if constexpr (K == 1) {
      // ---- DC only (r = 1).  The kept coefficient is the block sum Y[0][0]
      // (row 0 of T is all ones), and the inverse of a lone DC is the
      // constant W_0^2 Y[0][0] = 9 Y_c[0][0] + 2304 * 128 at every pixel, an
      // integer below 2^24: the value the pruned passes form, rounded by the
      // same two multiplies.  Each lane sums its two rows of blocks p and
      // p + 4 (dp4a against ones, each partial < 2^13), the 8 lanes of a block
      // pair add them up as two 16-bit halves of one word (totals < 2^16).
      unsigned s2 = 0u;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        s2 = __dp4a(X[k].x, 0x01010101u, s2);
        s2 = __dp4a(X[k].y, 0x01010101u, s2);
        s2 = __dp4a(X[k].z, 0x01010101u, s2);
        s2 = __dp4a(X[k].w, 0x01010101u, s2);
      }
      unsigned sb = 0u;
#pragma unroll
      for (int k = 2; k < 4; ++k) {
        sb = __dp4a(X[k].x, 0x01010101u, sb);
        sb = __dp4a(X[k].y, 0x01010101u, sb);
        sb = __dp4a(X[k].z, 0x01010101u, sb);
        sb = __dp4a(X[k].w, 0x01010101u, sb);
      }
      s2 |= sb << 16;
      s2 += __shfl_xor_sync(0xffffffffu, s2, 4);
      s2 += __shfl_xor_sync(0xffffffffu, s2, 8);
      s2 += __shfl_xor_sync(0xffffffffu, s2, 16);
      const int ya = (int)(s2 & 0xffffu) - 32768, yb = (int)(s2 >> 16) - 32768;  // Y_c[0][0], blocks p, p + 4

      have_fut = hq[D - 1] && ok && c_t < t_stop;  // the input rows of the tile D ahead
      if (have_fut) {
        take(fut);
        ok = advance();
        issue(fut, st);
      } else {
        cp_async_commit();
      }

      const unsigned qa = round_dc(__fmaf_rn((float)ya, 9.0f, 294912.0f));
      const unsigned qb = round_dc(__fmaf_rn((float)yb, 9.0f, 294912.0f));
      const unsigned wa = pack_u8(qa, qa, pack_u8(qa, qa, 0u)), wb = pack_u8(qb, qb, pack_u8(qb, qb, 0u));
#pragma unroll
      for (int tr = 0; tr < 2; ++tr) {
        uint8_t* d = cur.dst + tr * cur.dst_pitch;
        if (va) __stcs(reinterpret_cast<uint4*>(d), make_uint4(wa, wa, wa, wa));
        if (vb) __stcs(reinterpret_cast<uint4*>(d + 64), make_uint4(wb, wb, wb, wb));
      }
      if (j == 0) {  // the kept energy W_0^2 Y_c^2, once per block pair
        ke = (unsigned long long)(unsigned)(ya * ya) * 9ull + (unsigned long long)(unsigned)(yb * yb) * 9ull;
        dc_term = (long long)ya + yb;
      }
    } else {
    // ---- the row pass
    {
      Swar16 rv[2][16];
      row_pass(X, rv);
      uint2* const t1w = reinterpret_cast<uint2*>(t1 + p * kBoxT1Words + 2 * j);
#pragma unroll
      for (int c = 0; c < K; ++c) t1w[10 * c] = make_uint2(rv[0][c].v, rv[1][c].v);
    }
    __syncwarp();

    // ---- the input rows of the tile D ahead, into the slot just read
    have_fut = hq[D - 1] && ok && c_t < t_stop;
    if (have_fut) {
      take(fut);
      ok = advance();
      issue(fut, st);
    } else {
      cp_async_commit();
    }

    // ---- column pass on column c = j, exact scaled coefficients, kept
    // energy, inverse column pass into the back-transpose (columns c < K)
    {
      ZF2 y[16];
      Swar16 cw[16], yw[16];
      const uint4* const t1r = reinterpret_cast<const uint4*>(t1 + p * kBoxT1Words + 20 * j);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 v = t1r[q];
        cw[4 * q].v = v.x;
        cw[4 * q + 1].v = v.y;
        cw[4 * q + 2].v = v.z;
        cw[4 * q + 3].v = v.w;
      }
      fwd16(cw, yw);  // only the outputs u < K are used
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        if (u < K) {
          const float2 f = swar16_f2(yw[u].v);  // 2^23 + Y_c + 32768, blocks p and p + 4
          // -w (2^23 + 32768) (+ 2304 * 128 on the DC of column 0), exact: w 257 2^15 and 9 2^23
          const float kc = __fmaf_rn(kwf[u], -8421376.0f, (u == 0 && j == 0) ? 294912.0f : 0.0f);
          y[u].v = make_float2(__fmaf_rn(f.x, kwf[u], kc), __fmaf_rn(f.y, kwf[u], kc));
          y[u].z = false;
          const int ya = (int)(__float_as_uint(f.x) - 0x4B008000u), yb = (int)(__float_as_uint(f.y) - 0x4B008000u);
          ke += (unsigned long long)(unsigned)(ya * ya) * kwi[u];
          ke += (unsigned long long)(unsigned)(yb * yb) * kwi[u];
          if (u == 0) dc_term = (long long)ya + yb;
        } else {
          y[u].v = make_float2(0.f, 0.f);
          y[u].z = true;
        }
      }
      ZF2 uo[16];
      inv16(y, uo);
      if (j < K) {
        float4* const t2w = reinterpret_cast<float4*>(t2 + p * kBoxT2Units + 18 * j);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          t2w[q] = make_float4(uo[2 * q].v.x, uo[2 * q].v.y, uo[2 * q + 1].v.x, uo[2 * q + 1].v.y);
      }
    }
    __syncwarp();

    // ---- inverse row pass on rows 2j, 2j+1 -> exact Z, round, clamp, store
    {
      ZF2 v0[16], v1[16];
      const float4* const t2r = reinterpret_cast<const float4*>(t2 + p * kBoxT2Units + 2 * j);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        if (c < K) {
          const float4 v = t2r[9 * c];  // rows 2j, 2j+1 of column c
          v0[c] = ZF2{make_float2(v.x, v.y), false};
          v1[c] = ZF2{make_float2(v.z, v.w), false};
        } else {
          v0[c] = ZF2{make_float2(0.f, 0.f), true};
          v1[c] = v0[c];
        }
      }
#pragma unroll
      for (int tr = 0; tr < 2; ++tr) {
        ZF2 z[16];
        if (tr == 0) inv16(v0, z);
        else inv16(v1, z);
        unsigned oa[4], ob[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          unsigned qa[4], qb[4];
#pragma unroll
          for (int e4 = 0; e4 < 4; ++e4) {
            const float2 e = rne_denormal(f2mul(z[4 * g + e4].v, kInv2304));
            qa[e4] = __float_as_uint(e.x);
            qb[e4] = __float_as_uint(e.y);
          }
          oa[g] = pack_u8(qa[1], qa[0], pack_u8(qa[3], qa[2], 0u));
          ob[g] = pack_u8(qb[1], qb[0], pack_u8(qb[3], qb[2], 0u));
        }
        uint8_t* d = cur.dst + tr * cur.dst_pitch;
        if (va) __stcs(reinterpret_cast<uint4*>(d), make_uint4(oa[0], oa[1], oa[2], oa[3]));
        if (vb) __stcs(reinterpret_cast<uint4*>(d + 64), make_uint4(ob[0], ob[1], ob[2], ob[3]));
      }
    }

    }  // K > 1

    // ---- the tile's exact 2304 SSE: 2304 sum (x - 128)^2 - kept energy.  Per
    // block sum (x - 128)^2 = sum x^2 - 256 Y_c[0][0] - 4194304; lane (p, 0)
    // holds Y_c[0][0] of blocks p and p + 4.
    long long nume = (long long)ex;
    if (j == 0) nume -= 256 * dc_term + 2 * 4194304LL;
    nume = 2304 * nume - (long long)ke;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nume += __shfl_xor_sync(0xffffffffu, nume, o);
    if (lane == 0) tile_sse[cur.t] = (float)nume * (1.0f / 2304.0f);
    __syncwarp();  // buffer reads done before the next tile's writes

    if (!(D > 1 ? hq[D > 1 ? 1 : 0] : have_fut)) break;
#pragma unroll
    for (int i = 0; i + 1 < D; ++i) {
      q[i] = q[i + 1];
      hq[i] = hq[i + 1];
    }
    q[D - 1] = fut;
    hq[D - 1] = have_fut;
    st = st + 1 == D ? 0 : st + 1;
  }
  cp_async_wait<0>();
  if (!ok && lane == 0) set_status(status, kDevBadJob);
  pdl_chain_exit();  // the next kernel (or the PSNR finalize) may now take this CTA's place
}

template <int K, int D>
static cudaError_t launch_box_shape(const BoxConfig& bc, const ImageJob* d_jobs, int njobs, long long ntiles,
                                    const float2* d_wtab, float* d_tile_sse, int* d_status, int num_sms,
                                    cudaStream_t stream, bool dependent, bool early) {
  const int threads = 32 * bc.warps, smem = bc.warps * box_warp_smem(D);
  int per_sm = 0;
  cudaError_t e = cudaFuncSetAttribute(zonal_box_kernel<K, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zonal_box_kernel<K, D>, threads, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, per_sm);
  const int ctas = bc.ctas_per_sm > 0 ? std::min(bc.ctas_per_sm, per_sm) : per_sm;
  const long long need = (ntiles + bc.warps - 1) / bc.warps;
  const int grid = (int)std::max<long long>(1, std::min<long long>((long long)num_sms * ctas, need));
  return launch_chained(zonal_box_kernel<K, D>, grid, threads, smem, stream, dependent, d_jobs, njobs, ntiles, d_wtab,
                        d_tile_sse, d_status, early ? 1 : 0, bc.vec);
}

bool box_config_supported(const BoxConfig& bc) {
  return (bc.warps == 2 || bc.warps == 4 || bc.warps == 8) && (bc.depth >= 1 && bc.depth <= 3) &&
         (bc.vec == 8 || bc.vec == 16) && bc.ctas_per_sm >= 0;
}

// The autotuner's choice on the 64 x 512^2 x 8 r workload (GB300): eight
// warps per CTA, one CTA per SM, input rows one tile ahead; with half the
// warps resident each warp walks twice the tiles, which amortises its start
// (job search, first copies) -- 84.9 us against 89.9 us at full occupancy.
BoxConfig default_box_config() { return BoxConfig{8, 1, 16, 1}; }

int box_config_max_ctas_per_sm(const BoxConfig& bc) {
  int n = 0;
  const int threads = 32 * bc.warps, smem = bc.warps * box_warp_smem(bc.depth);
  cudaError_t e = cudaSuccess;
  switch (bc.depth) {
    case 1:
      e = cudaFuncSetAttribute(zonal_box_kernel<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zonal_box_kernel<8, 1>, threads, smem);
      break;
    case 3:
      e = cudaFuncSetAttribute(zonal_box_kernel<8, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zonal_box_kernel<8, 3>, threads, smem);
      break;
    default:
      e = cudaFuncSetAttribute(zonal_box_kernel<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zonal_box_kernel<8, 2>, threads, smem);
  }
  return (e == cudaSuccess && n > 0) ? n : 1;
}

// The box kernel of extent K in shape bc.  The staging depth is a tuning
// knob of the K = 8 kernel (the extent of r <= 36, config-4-like batches);
// the other extents run with depth 2.
template <int K>
static cudaError_t launch_box(const BoxConfig& bc, const ImageJob* d_jobs, int njobs, long long ntiles,
                              const float2* d_wtab, float* d_tile_sse, int* d_status, int num_sms,
                              cudaStream_t stream, bool dependent, bool early) {
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles >= (1LL << 30) || !box_config_supported(bc)) return cudaErrorInvalidValue;
  if constexpr (K == 8) {
    if (bc.depth == 1)
      return launch_box_shape<K, 1>(bc, d_jobs, njobs, ntiles, d_wtab, d_tile_sse, d_status, num_sms, stream,
                                    dependent, early);
    if (bc.depth == 3)
      return launch_box_shape<K, 3>(bc, d_jobs, njobs, ntiles, d_wtab, d_tile_sse, d_status, num_sms, stream,
                                    dependent, early);
  }
  return launch_box_shape<K, 2>(bc, d_jobs, njobs, ntiles, d_wtab, d_tile_sse, d_status, num_sms, stream,
                                dependent, early);
}

// --------------------------------------------------------------------------
// Host: classes of zonal jobs.
// --------------------------------------------------------------------------
int zonal_class_of(int r) {
  for (int c = 0; c < kZonalBoxClasses; ++c)
    if (r >= 1 && r <= box_max_r(kZonalBoxK[c])) return c;
  return kZonalGeneral;
}

void zonal_order(const ImageJob* jobs, int n, ImageJob* ordered, ZonalSplit* split) {
  int count[kZonalClasses] = {0};
  for (int i = 0; i < n; ++i) ++count[zonal_class_of(jobs[i].param)];
  split->first[0] = 0;
  for (int c = 0; c < kZonalClasses; ++c) split->first[c + 1] = split->first[c] + count[c];
  int pos[kZonalClasses];
  for (int c = 0; c < kZonalClasses; ++c) {
    pos[c] = split->first[c];
    split->ntiles[c] = 0;
  }
  for (int i = 0; i < n; ++i) {
    const int c = zonal_class_of(jobs[i].param);
    ImageJob J = jobs[i];
    const long long tiles = (long long)J.tiles_x * (J.height / kTileH);
    J.level_base = J.tile_begin;  // where this job's per-tile partials go
    J.tile_begin = split->ntiles[c];
    split->ntiles[c] += tiles;
    ordered[pos[c]++] = J;
  }
}

cudaError_t launch_zonal_ordered(const ImageJob* d_ordered, const ZonalSplit& split, const ZonalConfig& general,
                                 int general_grid, const BoxConfig& box, const float2* d_wtab, float* d_tile_sse,
                                 int* d_status, int num_sms, cudaStream_t stream) {
  // The general class first (the longest), then the box classes from the
  // largest extent down; every launch after the first is a programmatic
  // dependent launch whose CTAs take the places of its predecessor's as they
  // retire, and every kernel but the last lets its successor be scheduled
  // from its start.
  static constexpr int kOrder[kZonalClasses] = {kZonalGeneral, 3, 2, 1, 0};
  int last = -1;
  for (int k = 0; k < kZonalClasses; ++k)
    if (split.first[kOrder[k] + 1] > split.first[kOrder[k]] && split.ntiles[kOrder[k]] > 0) last = k;
  cudaError_t e = cudaSuccess;
  bool dependent = false;
  for (int k = 0; k < kZonalClasses && e == cudaSuccess; ++k) {
    const int c = kOrder[k];
    const int nj = split.first[c + 1] - split.first[c];
    if (nj == 0 || split.ntiles[c] == 0) continue;
    const ImageJob* jobs = d_ordered + split.first[c];
    const long long nt = split.ntiles[c];
    const bool early = k != last;
    switch (c) {
      case 0: e = launch_box<1>(box, jobs, nj, nt, d_wtab, d_tile_sse, d_status, num_sms, stream, dependent, early); break;
      case 1: e = launch_box<3>(box, jobs, nj, nt, d_wtab, d_tile_sse, d_status, num_sms, stream, dependent, early); break;
      case 2: e = launch_box<6>(box, jobs, nj, nt, d_wtab, d_tile_sse, d_status, num_sms, stream, dependent, early); break;
      case 3: e = launch_box<8>(box, jobs, nj, nt, d_wtab, d_tile_sse, d_status, num_sms, stream, dependent, early); break;
      default: {
        const long long need = (nt + general.warps - 1) / general.warps;
        const int grid = (int)std::max<long long>(1, std::min<long long>(general_grid, need));
        e = launch_zonal_config(general, jobs, nj, nt, d_wtab, d_tile_sse, d_status, grid, stream, dependent, early);
      }
    }
    dependent = true;
  }
  return e;
}

}  // namespace atdct16
