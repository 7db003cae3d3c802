// sm_103a kernels for the 16x16 multiplierless transform of arXiv 1606.05562.
//
// Work decomposition shared by the fused kernels
// ----------------------------------------------
// A warp owns one 16 x 128 tile (eight 16x16 blocks) at a time and walks the
// tiles of a whole batch in a persistent loop.  Inside the warp, lane
// l = 8 p + j works on the block pair (A, B) = (block p, block p + 4) of the
// tile.  Every value is a packed float2 holding the same position of blocks A
// and B, so each f32x2 instruction advances both blocks.
//   row pass      : lane j holds image rows 2j, 2j+1 of A and B
//   transpose     : through a warp-private 8 KB shared-memory buffer,
//                   XOR-swizzled on 16-byte chunks (conflict-free both ways)
//   column pass   : lane j holds columns 2j, 2j+1 of A and B
//   scale / mask  : per coefficient, weights from a per-r table
//   inverse column, transpose back, inverse row, round, store.
//
// Exactness.  u8 pixels enter as 2^23 + 256 x (one byte permute builds the
// float); every forward node is then a multiple of 256 below 2^32, so the
// integer transform Y = T X T^T is exact in FP32.  The zonal inverse works on
// the integers D = keep * W_u W_v Y (W = 48 S^2 in {3, 4, 6}) and produces the
// integer numerator Z = T^T D T of X_hat = Z / 2304; every intermediate stays
// below 2^24 for all zig-zag prefixes and u8 input, so Z is exact too.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "atdct16_butterfly.cuh"
#include "atdct16_device.cuh"
#include "atdct16_internal.h"
#include "atdct16_zigzag.cuh"

#include <atomic>
#include <cmath>
#include <type_traits>

namespace atdct16 {

// --------------------------------------------------------------------------
// Fused zonal compression: forward, keep the first r zig-zag coefficients,
// S^2 scaling, inverse, round, store u8, per-tile SSE (Sec. 4 procedure).
//
// Lane (p, j) = (lane & 3, lane >> 2) owns rows 2j, 2j+1 of blocks p and
// p + 4 of a 16 x 128 tile (the two blocks ride in the two halves of each
// register), so each quarter-warp touches two 64-byte row segments per
// global access.
//
// The forward transform is exact integer work.  The row pass runs on the
// integer pipe, two blocks per 32-bit word (one 3-operand add per butterfly
// addition).  The column pass runs either there too (kColSwar: int16
// fields; the row pass centres its DC output by -2048, which keeps every
// column node inside int16: |row outputs| <= 4080, column nodes within
// [-32768, 32640]) and a byte permute plus one exact FMA turn each
// coefficient field into the float 256 Y; or on f32x2 from 13-bit row
// fields that a byte permute places into float mantissas.  The mask, the
// S^2 weights, the dropped energy and the inverse run on f32x2.
//
// Shared memory per warp, in 16-byte units (padded, so that every access is
// a per-lane base plus a compile-time offset, and conflict-free), plus two
// staging slots for the input rows of the next two tiles:
//   back-transpose   unit(p, c, q) = 138 p + 8 c + (c >> 1) + q: rows 2q,
//                    2q+1 of column c of block pair p (549 units);
//   forward transpose: the chunk with columns 2cc, 2cc+1 of rows 2q, 2q+1
//                    sits at unit(p, 2cc + (1 ^ ((cc >> 1) & 1)), q), in the
//                    line of the column that its only reader, lane (p, cc),
//                    writes last, after it has read the whole chunk;
//   weights          unit(c, h) = 549 + 9 c + h (143 units).
// The input rows of the tile after next are copied in while a tile is computed.
// --------------------------------------------------------------------------
constexpr int kZT2Units = 549;
constexpr int kZWUnits = 143;
constexpr int kZStageUnits = 2 * 4 * 32;  // two tiles of input rows, 4 x 16 bytes per lane
constexpr int kZonalWarpSmemBytes = 16 * (kZT2Units + kZWUnits + kZStageUnits);

template <int kWarps, bool kColSwar>
__global__ void __launch_bounds__(32 * kWarps, 12 / kWarps)
zonal_f32_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles_ll,
             const float2* __restrict__ wtab, float* __restrict__ tile_sse, int* __restrict__ status,
             int pdl_early) {
  extern __shared__ __align__(16) unsigned char zsmem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane & 3, j = lane >> 2, jb1 = (j >> 1) & 1;
  float4* const t2 = reinterpret_cast<float4*>(zsmem + warp * kZonalWarpSmemBytes);
  float4* const wsm = t2 + kZT2Units;
  uint4* const stg = reinterpret_cast<uint4*>(wsm + kZWUnits) + lane;  // + 128 s + 32 k
  const int ntiles = (int)ntiles_ll;  // the launcher checks ntiles < 2^31
  // row-pass words: 13-bit fields (bias 4096) for a float column pass,
  // int16 fields (bias 32768) for an integer one
  using Row = typename std::conditional<kColSwar, Swar16, SwarRow>::type;
  constexpr unsigned kRowBias = kColSwar ? kSwarBias : kSwarRowBias;

  // Each warp takes a contiguous range of tiles and walks it with a cursor:
  // one job lookup per image, then the tile column/band advance by addition.
  const int nwarps = gridDim.x * kWarps;
  const int per_warp = (ntiles + nwarps - 1) / nwarps;
  const int t_first = (blockIdx.x * kWarps + warp) * per_warp;
  const int t_stop = min(ntiles, t_first + per_warp);
  if (pdl_early) pdl_launch_dependents();  // the next class's kernel may be scheduled
  if (t_first >= t_stop) {
    pdl_chain_exit();
    return;
  }

  int c_t = 0, c_end = 0, tiles_x = 1, tx = 0, nb_last = 8, r_job = 0, src_pitch = 0, dst_pitch = 0, t_shift = 0;
  const uint8_t* src_band = nullptr;  // this lane's row 2j of block p in tile column 0 of the band
  uint8_t* dst_band = nullptr;
  auto enter = [&](int t) -> bool {   // place the cursor on tile t
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
    t_shift = (int)(__ldg(&J->level_base) - (long long)(t - lt));  // partials: level_base + (t - tile_begin)
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
  auto take = [&](ZonalTile& z) {     // the cursor's tile
    z.src = src_band + tx * kTileW;
    z.dst = dst_band + tx * kTileW;
    z.src_pitch = src_pitch;
    z.dst_pitch = dst_pitch;
    z.nb = tx == tiles_x - 1 ? nb_last : 8;
    z.t = c_t + t_shift;
    z.r = r_job;
  };
  auto advance = [&]() -> bool {      // false: the job table does not cover the next tile
    ++c_t;
    if (++tx == tiles_x) {
      tx = 0;
      src_band += (long long)kTileH * src_pitch;
      dst_band += (long long)kTileH * dst_pitch;
    }
    return c_t >= t_stop || c_t < c_end || enter(c_t);
  };
  // Input rows of tile z into staging slot st: word k = row 2j + (k & 1) of
  // block p + 4 (k >> 1).  Each lane reads back only what it copied itself.
  // Blocks past the image edge are not copied; their stale words are finite
  // bytes whose results are never stored.
  auto issue = [&](const ZonalTile& z, int st) {
    uint4* d = stg + 128 * st;
    if (p < z.nb) {
      cp_async16(d, z.src);
      cp_async16(d + 32, z.src + z.src_pitch);
    }
    if (p + 4 < z.nb) {
      cp_async16(d + 64, z.src + 64);
      cp_async16(d + 96, z.src + 64 + z.src_pitch);
    }
    cp_async_commit();
  };

  if (!enter(t_first)) {
    if (lane == 0) set_status(status, kDevBadJob);
    pdl_chain_exit();
    return;
  }
  int wr = -1;  // r whose weights are in wsm
  bool ok = true;

  ZonalTile cur, nxt;
  take(cur);
  ok = advance();
  issue(cur, 0);
  bool have_nxt = ok && c_t < t_stop;
  if (have_nxt) {
    take(nxt);
    ok = advance();
    issue(nxt, 1);
  } else {
    cp_async_commit();
  }
  int st = 0;
  while (true) {
    // ---- this tile's input rows (copied one or two tile times ago)
    cp_async_wait<1>();
    uint4 X[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) X[k] = stg[128 * st + 32 * k];
    const bool va = p < cur.nb, vb = p + 4 < cur.nb;
    if (cur.r != wr) {  // warp-uniform: refresh the weight copy
      __syncwarp();
      const float4* src = reinterpret_cast<const float4*>(wtab) + (long long)cur.r * 128;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int g = lane * 4 + q;
        wsm[9 * (g >> 3) + (g & 7)] = __ldg(src + g);  // (kw, dw) of rows 2h, 2h + 1 of column g >> 3
      }
      __syncwarp();
      wr = cur.r;
    }

    // ---- row pass (Sec. 2 factorisation), exact, two blocks per word
    {
      Row rv[2][16];
#pragma unroll
      for (int tr = 0; tr < 2; ++tr) {
        const uint4& wa = X[tr];
        const uint4& wb = X[2 + tr];
        Row xs[16];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const unsigned lo = __byte_perm(word_of(wa, w), word_of(wb, w), 0x5410u);  // a0 a1 b0 b1
          const unsigned hi = __byte_perm(word_of(wa, w), word_of(wb, w), 0x7632u);  // a2 a3 b2 b3
          xs[4 * w + 0].v = (lo & 0x00FF00FFu) | kRowBias;
          xs[4 * w + 1].v = __byte_perm(lo, kRowBias, 0x7351u);
          xs[4 * w + 2].v = (hi & 0x00FF00FFu) | kRowBias;
          xs[4 * w + 3].v = __byte_perm(hi, kRowBias, 0x7351u);
        }
        fwd16(xs, rv[tr]);
        if (kColSwar) rv[tr][0].v -= 0x08000800u;  // centre the DC output by -2048
      }
      uint4* const t1w = reinterpret_cast<uint4*>(t2 + 138 * p + j);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc)
        t1w[17 * cc + 8 * (1 ^ ((cc >> 1) & 1))] =
            make_uint4(rv[0][2 * cc].v, rv[1][2 * cc].v, rv[0][2 * cc + 1].v, rv[1][2 * cc + 1].v);
    }
    __syncwarp();

    // ---- the input rows of the tile after the next one, into the slot
    // that X came from (X is consumed)
    ZonalTile fut;
    const bool have_fut = have_nxt && ok && c_t < t_stop;
    if (have_fut) {
      take(fut);
      ok = advance();
      issue(fut, st);
    } else {
      cp_async_commit();
    }

    // ---- per column c = 2j + i: column pass (y = 256 Y, exact), mask and S^2
    // weights, dropped energy (Parseval), inverse column pass into the
    // back-transpose.  Lanes with odd j >> 1 take their two columns in the
    // opposite order, so the 8-byte reads of the forward transpose are
    // conflict-free; each lane's forward chunks sit in the line it writes last.
    float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    const uint2* const t1r = reinterpret_cast<const uint2*>(t2 + 138 * p + 17 * j + 8 * (1 ^ jb1));
#pragma unroll
    for (int ii = 0; ii < 2; ++ii) {
      const int i = ii ^ jb1;
      float2 y[16];
      if constexpr (kColSwar) {
        Swar16 cw[16], yw[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint2 v = t1r[2 * q + i];
          cw[2 * q].v = v.x;
          cw[2 * q + 1].v = v.y;
        }
        fwd16(cw, yw);
        // field f -> float 2^23 + f (f = Y + 32768) -> 256 f - 256 (2^23 +
        // 32768) = 256 Y in one exact FMA; the DC coefficient of column 0
        // also takes back the 16 * 2048 of the centring
        const float dc = (2 * j + i) == 0 ? -2147483648.0f : -2155872256.0f;
#pragma unroll
        for (int u = 0; u < 16; ++u) {  // scalar FMAs: immediate operands, no constant pairs to hold
          const float o = u == 0 ? dc : -2155872256.0f;
          const float2 f = swar16_f2(yw[u].v);
          y[u] = make_float2(__fmaf_rn(f.x, 256.0f, o), __fmaf_rn(f.y, 256.0f, o));
        }
      } else {
        float2 cv[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint2 v = t1r[2 * q + i];
          cv[2 * q] = swar_row_f2(v.x);
          cv[2 * q + 1] = swar_row_f2(v.y);
        }
        fwd16(cv, y);
        // every input carries 2^23 + 2^20; only the DC row sums them
        y[0] = bsub(y[0], make_float2(150994944.0f, 150994944.0f));
      }
      const float4* const wcol = wsm + 9 * (2 * j + i);
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const float4 w = wcol[h];
        acc = __ffma2_rn(f2mul(y[2 * h], w.y), y[2 * h], acc);
        acc1 = __ffma2_rn(f2mul(y[2 * h + 1], w.w), y[2 * h + 1], acc1);
        y[2 * h] = f2mul(y[2 * h], w.x);
        y[2 * h + 1] = f2mul(y[2 * h + 1], w.z);
      }
      float2 uo[16];
      inv16(y, uo);
      float4* const t2w = t2 + 138 * p + 17 * j + 8 * i;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        t2w[q] = make_float4(uo[2 * q].x, uo[2 * q].y, uo[2 * q + 1].x, uo[2 * q + 1].y);
    }
    __syncwarp();

    // ---- per row 2j + rr: gather the row (8-byte halves of the chunks),
    // inverse row pass -> exact Z, round half to even, clamp, pack, store.
    // Lanes with odd j >> 1 take their two rows in the opposite order: the
    // lanes of a half-warp that meet on a chunk position then read its two
    // different halves (conflict-free), while a quarter-warp still stores
    // two whole 64-byte row segments.
#pragma unroll
    for (int tr = 0; tr < 2; ++tr) {
      const int rr = tr ^ jb1;
      const float2* const fin = reinterpret_cast<const float2*>(t2 + 138 * p + j) + rr;
      float2 v[16], z[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = fin[2 * (8 * c + (c >> 1))];
      inv16(v, z);
      unsigned oa[4], ob[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        unsigned qa[4], qb[4];
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
          const float2 e = rne_denormal(f2mul(z[4 * g + e4], kInv2304));
          qa[e4] = __float_as_uint(e.x);
          qb[e4] = __float_as_uint(e.y);
        }
        oa[g] = pack_u8(qa[1], qa[0], pack_u8(qa[3], qa[2], 0u));
        ob[g] = pack_u8(qb[1], qb[0], pack_u8(qb[3], qb[2], 0u));
      }
      uint8_t* d = cur.dst + rr * cur.dst_pitch;
      if (va) __stcs(reinterpret_cast<uint4*>(d), make_uint4(oa[0], oa[1], oa[2], oa[3]));
      if (vb) __stcs(reinterpret_cast<uint4*>(d + 64), make_uint4(ob[0], ob[1], ob[2], ob[3]));
    }

    // ---- tile SSE: dropped energy / (256 * 2304), summed over valid blocks
    acc = __fadd2_rn(acc, acc1);
    const float tot = warp_sum((va ? acc.x : 0.f) + (vb ? acc.y : 0.f));
    if (lane == 0) tile_sse[cur.t] = tot * (1.0f / (256.0f * 2304.0f));
    __syncwarp();  // buffer reads done before the next tile's writes

    if (!have_nxt) break;
    cur = nxt;
    nxt = fut;
    have_nxt = have_fut;
    st ^= 1;
  }
  cp_async_wait<0>();
  if (!ok && lane == 0) set_status(status, kDevBadJob);
  pdl_chain_exit();  // the next kernel (or the PSNR finalize) may now take this CTA's place
}

// --------------------------------------------------------------------------
// Fused zonal compression with the forward transform on the tensor cores.
//
// The 2-D forward transform of a block is two exact 16x16 integer products,
// P = T X and Y = P T^T, and both run as m16n8k16 f16 MMAs with FP32
// accumulation: X enters as the f16 values 1024 + x (one byte permute per
// pair, straight from an ldmatrix.trans of the staged rows, which hands each
// lane the B-operand pairs (rows 2q, 2q+1) of pixel columns 2g and 2g+1);
// P's DC row is centred through the accumulator initialisation
// (-16384 - 2048), so every entry of P lies in [-2048, 2040] and is exact in
// f16; P's accumulator fragments are the A operand of the second product
// (its column order is absorbed into a permuted constant T^T), whose
// accumulator starts at +32768 on Y[0][0] to undo the centring.  All
// products are integers below 2^24: Y is exact.
//
// Each lane then holds Y at the fixed positions (u, v) = (g, 2q..2q+1),
// (g+8, ...), (g, 8+2q..), (g+8, 8+2q..) of every block (g = lane >> 2,
// q = lane & 3), so the zonal weights of the warp's current r live in
// registers (as f32x2 pairs over v, v+1).  The masked, weighted V goes to
// the back-transpose buffer as (block p, block p+4) pairs; the inverse
// column and row passes, the exact rounding and the stores are those of the
// integer-pipe kernel.
//
// Shared memory per warp (13.4 KB): the back-transpose
// unit(p, c, q) = R(p) + 8 c + (c & 14) + q, R = (0, 145, 292, 437)
// (16-byte units, 579 of them), conflict-free for the MMA-side 8-byte
// writes, the column pass's 16-byte reads and writes and the row pass's
// 8-byte reads (lanes with odd j take their two rows in reverse order); and
// two staging slots of 16 rows x 16 bytes per block, row r of block b at
// 16 b + (r ^ x(b & 3)), x = (0, 1, 4, 5): conflict-free for the cp.async
// writes and the ldmatrix reads.
// --------------------------------------------------------------------------
constexpr int kMUnits = 579;
constexpr int kMStageUnits = 2 * 128;
constexpr int kZonalMmaWarpSmemBytes = 16 * (kMUnits + kMStageUnits);

__host__ __device__ constexpr int mma_region(int p) { return p == 0 ? 0 : (p == 1 ? 145 : (p == 2 ? 292 : 437)); }
__device__ __forceinline__ int stage_slot(int b, int r) {
  const int pb = b & 3;
  return 16 * b + (r ^ ((pb & 1) | ((pb & 2) << 1)));
}

__device__ __forceinline__ void ldsm_x4_trans(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
// D = A B + C, m16n8k16, A row-major f16, B column-major f16, C/D f32
__device__ __forceinline__ void mma_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1,
                                          const float (&c)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%10, %11, %12, %13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]),
        "f"(c[3]));
}
// (lo, hi) -> f16x2 with lo in the low half (exact for the integers used)
__device__ __forceinline__ unsigned pack_f16x2(float lo, float hi) {
  unsigned d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ unsigned f16_of_t(int t) { return t == 0 ? 0u : (t > 0 ? 0x3C00u : 0xBC00u); }
__device__ __forceinline__ unsigned f16x2_of_t(int lo, int hi) { return f16_of_t(lo) | (f16_of_t(hi) << 16); }

template <int kWarps>
__global__ void __launch_bounds__(32 * kWarps, 12 / kWarps)
zonal_mma_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles_ll,
                 const float2* __restrict__ wtab, float* __restrict__ tile_sse, int* __restrict__ status,
             int pdl_early) {
  extern __shared__ __align__(16) unsigned char msmem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;  // MMA fragment coordinates
  const int p = q, j = g;                 // back half: block pair p, row pair j
  float4* const tb = reinterpret_cast<float4*>(msmem + warp * kZonalMmaWarpSmemBytes);
  uint4* const stg = reinterpret_cast<uint4*>(tb + kMUnits);  // + 128 slot + stage_slot(b, r)
  const int ntiles = (int)ntiles_ll;  // the launcher checks ntiles < 2^30

  // ---- constant MMA operands from the Sec. 2 factorisation: columns of T
  // are the butterfly's responses to unit vectors
  unsigned ta[4], tbf[2][2];
  {
    // rows g and g + 8 of the columns k = 2q, 2q+1, 2q+8, 2q+9, 4q .. 4q+3
    int tg[8], tg8[8];
    const int ks[8] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9, 4 * q, 4 * q + 1, 4 * q + 2, 4 * q + 3};
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      int e[16], col[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) e[k] = k == ks[n] ? 1 : 0;
      fwd16(e, col);
      int a = 0, b8 = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        a = u == g ? col[u] : a;
        b8 = u == g ? col[u + 8] : b8;
      }
      tg[n] = a;
      tg8[n] = b8;
    }
    // stage 1, A = T (m = u, k = pixel row): rows g, g + 8; k = 2q, 2q+1, 2q+8, 2q+9
    ta[0] = f16x2_of_t(tg[0], tg[1]);
    ta[1] = f16x2_of_t(tg8[0], tg8[1]);
    ta[2] = f16x2_of_t(tg[2], tg[3]);
    ta[3] = f16x2_of_t(tg8[2], tg8[3]);
    // stage 2, B[k][v] = T[v][col(k)], col(2q) = 4q, col(2q+1) = 4q+2,
    // col(2q+8) = 4q+1, col(2q+9) = 4q+3; n = v = g (tile 0) or g + 8 (tile 1)
    tbf[0][0] = f16x2_of_t(tg[4], tg[6]);
    tbf[0][1] = f16x2_of_t(tg[5], tg[7]);
    tbf[1][0] = f16x2_of_t(tg8[4], tg8[6]);
    tbf[1][1] = f16x2_of_t(tg8[5], tg8[7]);
  }

  const int nwarps = gridDim.x * kWarps;
  const int per_warp = (ntiles + nwarps - 1) / nwarps;
  const int t_first = (blockIdx.x * kWarps + warp) * per_warp;
  const int t_stop = min(ntiles, t_first + per_warp);
  if (pdl_early) pdl_launch_dependents();  // the next class's kernel may be scheduled
  if (t_first >= t_stop) {
    pdl_chain_exit();
    return;
  }

  int c_t = 0, c_end = 0, tiles_x = 1, tx = 0, nb_last = 8, r_job = 0, src_pitch = 0, dst_pitch = 0, t_shift = 0;
  const uint8_t* src_band = nullptr;  // row 0 of the current band, tile column 0
  uint8_t* dst_band = nullptr;        // this lane's row 2j of block p in tile column 0 of the band
  auto enter = [&](int t) -> bool {
    int job;
    warp_find_job(jobs, njobs, t, job);
    const ImageJob* J = jobs + job;
    const long long tb0 = __ldg(&J->tile_begin);
    tiles_x = __ldg(&J->tiles_x);
    const long long te = tb0 + (long long)tiles_x * (__ldg(&J->height) >> 4);
    if (t < tb0 || t >= te || tiles_x < 1) return false;
    c_end = (int)min(te, (long long)t_stop);
    const int lt = (int)(t - tb0);
    const int ty = lt / tiles_x;
    tx = lt - ty * tiles_x;
    t_shift = (int)(__ldg(&J->level_base) - (long long)(t - lt));  // partials: level_base + (t - tile_begin)
    src_pitch = (int)__ldg(&J->src_pitch);
    dst_pitch = (int)__ldg(&J->dst_pitch);
    const long long row0 = (long long)ty * kTileH;
    src_band = reinterpret_cast<const uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->src))) +
               (row0 + 2 * j) * src_pitch + 16 * p;
    dst_band = reinterpret_cast<uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->dst))) +
               (row0 + 2 * j) * dst_pitch + 16 * p;
    nb_last = min(8, (__ldg(&J->width) - (tiles_x - 1) * kTileW) >> 4);
    r_job = __ldg(&J->param);
    c_t = t;
    return true;
  };
  auto take = [&](ZonalTile& z) {
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
  // Rows 2j, 2j+1 of blocks p and p+4 of tile z into staging slot st.
  // Blocks past the image edge are filled with zeros (nothing is read):
  // their coefficients and dropped energy are then exactly 0.
  auto issue = [&](const ZonalTile& z, int st) {
    uint4* const d = stg + 128 * st;
    const int na = p < z.nb ? 16 : 0, nb4 = p + 4 < z.nb ? 16 : 0;
    const uint8_t* sa = na ? z.src : z.src - 16 * p;  // a valid address either way
    const uint8_t* sb = nb4 ? z.src + 64 : sa;
    cp_async16_zfill(d + stage_slot(p, 2 * j), sa, na);
    cp_async16_zfill(d + stage_slot(p, 2 * j + 1), sa + (na ? z.src_pitch : 0), na);
    cp_async16_zfill(d + stage_slot(p + 4, 2 * j), sb, nb4);
    cp_async16_zfill(d + stage_slot(p + 4, 2 * j + 1), sb + (nb4 ? z.src_pitch : 0), nb4);
    cp_async_commit();
  };

  if (!enter(t_first)) {
    if (lane == 0) set_status(status, kDevBadJob);
    pdl_chain_exit();
    return;
  }
  bool ok = true;
  int wr = -1;
  // Zonal weights at this lane's coefficient positions, as f32x2 pairs over
  // (v, v+1): [nt][h] = rows u = g + 8 h, columns v = 8 nt + 2q, +1;
  // kw = keep W_u W_v, dw = (1 - keep) W_u W_v (the table holds them / 256)
  float2 kwp[2][2], dwp[2][2];
  const unsigned stg_base = (unsigned)__cvta_generic_to_shared(stg);
  // back-transpose bases of this lane: V writes (float2 units), column lines, row reads
  const int v_lane = 72 * q + 2 * g;
  const int rp = mma_region(p);
  // ldmatrix row address of this lane within a slot, for block pair b:
  // matrix (lane >> 3) = (block b + 4 (lane >> 4), rows 8 ((lane >> 3) & 1) ..)
  const int lrow = 8 * ((lane >> 3) & 1) + (lane & 7);
  // accumulator input of every MMA: four registers holding 0 (opaque, so they
  // are kept rather than rebuilt for each product)
  float zero4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) asm("mov.b32 %0, 0;" : "=f"(zero4[k]));
  const float2 i1 = g == 0 ? make_float2(-18432.0f, -18432.0f) : make_float2(0.f, 0.f);
  const float i2 = lane == 0 ? 32768.0f : 0.0f;

  ZonalTile cur, nxt;
  take(cur);
  ok = advance();
  issue(cur, 0);
  bool have_nxt = ok && c_t < t_stop;
  if (have_nxt) {
    take(nxt);
    ok = advance();
    issue(nxt, 1);
  } else {
    cp_async_commit();
  }
  int st = 0;
  while (true) {
    cp_async_wait<1>();
    __syncwarp();  // every lane's copies of this tile are visible to the warp
    if (cur.r != wr) {
      const float2* wr_tab = wtab + (long long)cur.r * 256;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int u = g + 8 * h, v = 8 * nt + 2 * q;
          const float2 w0 = __ldg(wr_tab + v * 16 + u), w1 = __ldg(wr_tab + (v + 1) * 16 + u);  // [r][c][u]
          kwp[nt][h] = make_float2(256.0f * w0.x, 256.0f * w1.x);
          dwp[nt][h] = make_float2(256.0f * w0.y, 256.0f * w1.y);
        }
      wr = cur.r;
    }

    // ---- forward transform of the eight blocks on the tensor cores, mask +
    // weights + dropped energy in registers, V into the buffer.  First the
    // row products of all eight blocks (independent MMAs back to back), then
    // the column products and the weighting, block pair by block pair.
    unsigned a2[4][2][4];  // [block pair][block b, b + 4][A fragment] of P, f16
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      unsigned x0, x1, x2, x3;  // blocks b (rows 0-7, 8-15), b + 4 (rows 0-7, 8-15)
      ldsm_x4_trans(stg_base + 16 * (128 * st + stage_slot(b + 4 * (lane >> 4), lrow)), x0, x1, x2, x3);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const unsigned lo = s ? x2 : x0, hi = s ? x3 : x1;
        // B operands: pixel column 2g (even tile) and 2g + 1 (odd tile), rows (2q, 2q+1), (2q+8, 2q+9)
        const unsigned be0 = __byte_perm(lo, 0x6464u, 0x4240u), be1 = __byte_perm(hi, 0x6464u, 0x4240u);
        const unsigned bo0 = __byte_perm(lo, 0x6464u, 0x4341u), bo1 = __byte_perm(hi, 0x6464u, 0x4341u);
        float pe[4], po[4];
        mma_16816(pe, ta, be0, be1, zero4);
        mma_16816(po, ta, bo0, bo1, zero4);
        // row u = 0 of P: remove 16 * 1024 and centre by -2048 (now |P| <= 2048)
        const float2 p0 = __fadd2_rn(make_float2(pe[0], pe[1]), i1), p1 = __fadd2_rn(make_float2(po[0], po[1]), i1);
        a2[b][s][0] = pack_f16x2(p0.x, p0.y);
        a2[b][s][1] = pack_f16x2(pe[2], pe[3]);
        a2[b][s][2] = pack_f16x2(p1.x, p1.y);
        a2[b][s][3] = pack_f16x2(po[2], po[3]);
      }
    }
    float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    float* const vdst = reinterpret_cast<float*>(tb) + v_lane;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      float yb[2][2][4];  // [block b, b + 4][nt][fragment]
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        mma_16816(yb[s][0], a2[b][s], tbf[0][0], tbf[0][1], zero4);
        mma_16816(yb[s][1], a2[b][s], tbf[1][0], tbf[1][1], zero4);
        yb[s][0][0] += i2;  // Y[0][0]: undo the centring
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 ya = make_float2(yb[0][nt][2 * h], yb[0][nt][2 * h + 1]);  // block b, (v, v+1)
          const float2 yB = make_float2(yb[1][nt][2 * h], yb[1][nt][2 * h + 1]);  // block b + 4
          acc = __ffma2_rn(__fmul2_rn(ya, dwp[nt][h]), ya, acc);
          acc1 = __ffma2_rn(__fmul2_rn(yB, dwp[nt][h]), yB, acc1);
          const float2 va2 = __fmul2_rn(ya, kwp[nt][h]), vb2 = __fmul2_rn(yB, kwp[nt][h]);
          // block b's value at word 0 and block b + 4's at word 1 of the pair
          // (u, v), u = g + 8h, v = 8 nt + 2q + e: float index
          // 4 unit(b, v, u >> 1) + 2 (u & 1) = 4 (R(b) + 72 nt + 8 e + 4 h) + 72 q + 2 g
          const int cu = 4 * (mma_region(b) + 72 * nt + 4 * h);
          vdst[cu] = va2.x;
          vdst[cu + 1] = vb2.x;
          vdst[cu + 32] = va2.y;
          vdst[cu + 33] = vb2.y;
        }
    }
    acc = __fadd2_rn(acc, acc1);
    __syncwarp();

    // ---- the input rows of the tile after the next one, into the slot just read
    ZonalTile fut;
    const bool have_fut = have_nxt && ok && c_t < t_stop;
    if (have_fut) {
      take(fut);
      ok = advance();
      issue(fut, st);
    } else {
      cp_async_commit();
    }

    // ---- per column c = 2j + i: inverse column pass, in place
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float4* const line = tb + rp + 18 * j + 8 * i;  // unit(p, 2j + i, 0)
      float2 y[16], uo[16];
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) {
        const float4 v = line[qq];
        y[2 * qq] = make_float2(v.x, v.y);
        y[2 * qq + 1] = make_float2(v.z, v.w);
      }
      inv16(y, uo);
#pragma unroll
      for (int qq = 0; qq < 8; ++qq)
        line[qq] = make_float4(uo[2 * qq].x, uo[2 * qq].y, uo[2 * qq + 1].x, uo[2 * qq + 1].y);
    }
    __syncwarp();

    // ---- per row 2j + rr: inverse row pass -> exact Z, round half to even,
    // clamp, pack, store (lanes with odd j take their rows in reverse order)
    const bool va = p < cur.nb, vb = p + 4 < cur.nb;
#pragma unroll
    for (int tr = 0; tr < 2; ++tr) {
      const int rr = tr ^ (j & 1);
      const float2* const fin = reinterpret_cast<const float2*>(tb + rp + j) + rr;
      float2 v[16], z[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = fin[2 * (8 * c + (c & 14))];
      inv16(v, z);
      unsigned oa[4], ob[4];
#pragma unroll
      for (int gg = 0; gg < 4; ++gg) {
        unsigned qa[4], qb[4];
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
          const float2 e = rne_denormal(f2mul(z[4 * gg + e4], kInv2304));
          qa[e4] = __float_as_uint(e.x);
          qb[e4] = __float_as_uint(e.y);
        }
        oa[gg] = pack_u8(qa[1], qa[0], pack_u8(qa[3], qa[2], 0u));
        ob[gg] = pack_u8(qb[1], qb[0], pack_u8(qb[3], qb[2], 0u));
      }
      uint8_t* d = cur.dst + rr * cur.dst_pitch;
      if (va) __stcs(reinterpret_cast<uint4*>(d), make_uint4(oa[0], oa[1], oa[2], oa[3]));
      if (vb) __stcs(reinterpret_cast<uint4*>(d + 64), make_uint4(ob[0], ob[1], ob[2], ob[3]));
    }

    // ---- tile SSE: dropped energy / 2304 (weights carry the 256)
    const float tot = warp_sum(acc.x + acc.y);
    if (lane == 0) tile_sse[cur.t] = tot * (1.0f / 2304.0f);
    __syncwarp();

    if (!have_nxt) break;
    cur = nxt;
    nxt = fut;
    have_nxt = have_fut;
    st ^= 1;
  }
  cp_async_wait<0>();
  if (!ok && lane == 0) set_status(status, kDevBadJob);
  pdl_chain_exit();  // the next kernel (or the PSNR finalize) may now take this CTA's place
}

// --------------------------------------------------------------------------
// Fused quantisation (S absorbed into the quantiser) for int16 planes
// (Sec. 2 last paragraph, Sec. 5.3).
//
// Same organisation as the zonal kernel: lane (p, j) = (lane & 3, lane >> 2)
// owns rows 2j, 2j+1 of blocks p and p + 4 of a 16 x 128-sample tile, input
// rows are staged with cp.async two tiles ahead, each warp walks a
// contiguous tile range with a cursor, and the transposes go through the
// padded line-per-column buffer unit(p, c, q) = 138 p + 8 c + (c >> 1) + q
// (the column pass overwrites, in place, the two lines each lane alone
// reads).  All arithmetic is FP32 on f32x2: int16 samples give exact
// integer Y (|Y| <= 2^23).  Per coefficient, with (k, s, g, Q) =
// (fp32(s_u s_v / Qstep), s_u s_v, s_u s_v Qstep, Qstep):
//   L  = floor(fp32(fp32(|Y| k) + 0.5))         (floor by a round-down add
//                                                of 2^23, exact for L < 2^22)
//   e  = s |Y| - L Q                             (B - B', Parseval)
//   Y' = sign(Y) L g                             (S B' S entry)
// and the reconstruction is rint to int16 (magic-number add, saturating pack).
// --------------------------------------------------------------------------
constexpr int kQStageUnits = 2 * 8 * 32;  // two tiles of input rows, 8 x 16 bytes per lane
constexpr int kQuantWarpSmemBytes = 16 * (kZT2Units + kQStageUnits);

// int16 field of a word -> 2^23 + 32768 + v as an exact float (offset binary
// placed in the mantissa): one logic op (low field) or a permute plus a logic
// op (high field), on the integer pipe.
__device__ __forceinline__ float i16_lo_m(unsigned w) { return __uint_as_float(((w & 0xffffu) ^ 0x8000u) | 0x4B000000u); }
__device__ __forceinline__ float i16_hi_m(unsigned w) {
  return __uint_as_float(__byte_perm(w, 0x4B00u, 0x5432u) ^ 0x8000u);
}

// a + b rounded toward -inf, both halves
__device__ __forceinline__ float2 f2add_rm(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(d);
}
// magnitude of m with the sign of s, both halves
__device__ __forceinline__ float2 f2copysign(float2 m, float2 s) {
  return make_float2(__uint_as_float((__float_as_uint(m.x) & 0x7fffffffu) | (__float_as_uint(s.x) & 0x80000000u)),
                     __uint_as_float((__float_as_uint(m.y) & 0x7fffffffu) | (__float_as_uint(s.y) & 0x80000000u)));
}

// Row u of T has nnz_u = 48 / W_u nonzeros: 16, 12 or 8 (class 0, 1, 2);
// quant_class_row gives one row of each class.
__host__ __device__ constexpr int quant_uclass(int u) {
  return (0x56945290u >> (2 * u)) & 3u;  // classes of u = 0..15: 0 0 1 2 2 0 1 1 0 1 1 2 2 1 1 1
}
__host__ __device__ constexpr int quant_class_row(int cl) { return cl == 0 ? 0 : (cl == 1 ? 2 : 3); }

struct QuantTile {
  const uint8_t* src;  // row 2j of block p of this lane
  uint8_t* dst;
  int src_pitch, dst_pitch;
  int nb;              // valid 16-sample blocks in the tile (1..8)
  int t;               // tile index
  int qp;
  long long lvl;       // level index of (u, v) = (0, 0) of block p of this tile
};

// Levels leave through the input staging slot of the current tile (free
// once its rows are in registers): the column pass writes the tile's 8 x 256
// int16 levels there in their output order, halfword k of block b at
// k ^ (16 (b & 3)), with k = 16 u + v row-major (conflict-free per-column
// writes) or k = the scan position of (u, v) when kZigzag (Sec. 4 scan; at
// most two lanes per bank), and the warp stores each block as one 512-byte
// run of 16-byte chunks.  The copy of the tile after next into that slot
// starts after the levels have left.
template <bool kLevels, bool kZigzag>
__global__ void __launch_bounds__(128, 3)
quant_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles_ll,
             const float4* __restrict__ qtab, int16_t* __restrict__ levels, float* __restrict__ tile_sse,
             int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char qsmem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane & 3, j = lane >> 2, jb1 = (j >> 1) & 1;
  float4* const tb = reinterpret_cast<float4*>(qsmem + warp * kQuantWarpSmemBytes);
  uint4* const stg = reinterpret_cast<uint4*>(tb + kZT2Units) + lane;  // + 256 s + 32 k
  const int ntiles = (int)ntiles_ll;  // the launcher checks ntiles < 2^30
  constexpr int kWarps = 4;
  const int nwarps = gridDim.x * kWarps;
  const int per_warp = (ntiles + nwarps - 1) / nwarps;
  const int t_first = (blockIdx.x * kWarps + warp) * per_warp;
  const int t_stop = min(ntiles, t_first + per_warp);
  if (t_first >= t_stop) return;

  int c_t = 0, c_end = 0, tiles_x = 1, tx = 0, ty = 0, nb_last = 8, qp_job = 0, src_pitch = 0, dst_pitch = 0;
  int bpr = 0;
  long long lvl_base = 0;
  const uint8_t* src_band = nullptr;  // this lane's row 2j of block p in tile column 0 of the band
  uint8_t* dst_band = nullptr;
  auto enter = [&](int t) -> bool {
    int job;
    warp_find_job(jobs, njobs, t, job);
    const ImageJob* J = jobs + job;
    const long long tb0 = __ldg(&J->tile_begin);
    tiles_x = __ldg(&J->tiles_x);
    const long long te = tb0 + (long long)tiles_x * (__ldg(&J->height) >> 4);
    if (t < tb0 || t >= te || tiles_x < 1) return false;
    c_end = (int)min(te, (long long)t_stop);
    const int lt = (int)(t - tb0);
    ty = lt / tiles_x;
    tx = lt - ty * tiles_x;
    src_pitch = (int)__ldg(&J->src_pitch);
    dst_pitch = (int)__ldg(&J->dst_pitch);
    const long long row = (long long)ty * kTileH + 2 * j;
    src_band = reinterpret_cast<const uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->src))) +
               row * src_pitch + 32 * p;
    dst_band = reinterpret_cast<uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->dst))) +
               row * dst_pitch + 32 * p;
    const int width = __ldg(&J->width);
    nb_last = min(8, (width - (tiles_x - 1) * kTileW) >> 4);
    bpr = width >> 4;
    lvl_base = __ldg(&J->level_base);
    qp_job = __ldg(&J->param);
    c_t = t;
    return true;
  };
  auto take = [&](QuantTile& z) {
    z.src = src_band + tx * (2 * kTileW);
    z.dst = dst_band + tx * (2 * kTileW);
    z.src_pitch = src_pitch;
    z.dst_pitch = dst_pitch;
    z.nb = tx == tiles_x - 1 ? nb_last : 8;
    z.t = c_t;
    z.qp = qp_job;
    z.lvl = lvl_base + ((long long)ty * bpr + tx * 8 + p) * 256;
  };
  auto advance = [&]() -> bool {
    ++c_t;
    if (++tx == tiles_x) {
      tx = 0;
      ++ty;
      src_band += (long long)kTileH * src_pitch;
      dst_band += (long long)kTileH * dst_pitch;
    }
    return c_t >= t_stop || c_t < c_end || enter(c_t);
  };
  // Staging word k of slot st: row 2j + ((k >> 1) & 1), block p + 4 (k >> 2),
  // samples 8 (k & 1) .. 8 (k & 1) + 7.
  auto issue = [&](const QuantTile& z, int st) {
    uint4* d = stg + 256 * st;
    if (p < z.nb) {
      cp_async16(d, z.src);
      cp_async16(d + 32, z.src + 16);
      cp_async16(d + 64, z.src + z.src_pitch);
      cp_async16(d + 96, z.src + z.src_pitch + 16);
    }
    if (p + 4 < z.nb) {
      cp_async16(d + 128, z.src + 128);
      cp_async16(d + 160, z.src + 144);
      cp_async16(d + 192, z.src + z.src_pitch + 128);
      cp_async16(d + 224, z.src + z.src_pitch + 144);
    }
    cp_async_commit();
  };

  if (!enter(t_first)) {
    if (lane == 0) set_status(status, kDevBadJob);
    return;
  }
  bool ok = true;
  QuantTile cur, nxt;
  take(cur);
  ok = advance();
  issue(cur, 0);
  bool have_nxt = ok && c_t < t_stop;
  if (have_nxt) {
    take(nxt);
    ok = advance();
    issue(nxt, 1);
  } else {
    cp_async_commit();
  }
  // Quantiser constants of the lane's two columns c = 2j + i: s_u s_v takes
  // one of three values per column (nnz_u in {16, 12, 8}), so k and g are
  // three register pairs per column, refreshed when the QP changes.
  int wq = -1;
  float kq[2][3], gq[2][3], qstep = 1.f;
  int st = 0;
  // scan positions of (u, 2j + i), one byte each: byte u & 3 of word 4 i + (u >> 2)
  unsigned zzl[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  if (kLevels && kZigzag) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int u = 0; u < 16; ++u) zzl[4 * i + (u >> 2)] |= (unsigned)zigzag_rank(16 * u + 2 * j + i) << (8 * (u & 3));
  }
  while (true) {
    cp_async_wait<1>();
    if (cur.qp != wq) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int cl = 0; cl < 3; ++cl) {
          const float4 q = __ldg(qtab + ((long long)cur.qp * 16 + 2 * j + i) * 16 + quant_class_row(cl));
          kq[i][cl] = q.x;
          gq[i][cl] = q.z;
          qstep = q.w;
        }
      wq = cur.qp;
    }
    uint4 X[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) X[k] = stg[256 * st + 32 * k];
    const bool va = p < cur.nb, vb = p + 4 < cur.nb;

    // ---- row pass on rows 2j, 2j+1 (exact), into the line-per-column buffer
    {
      float2* const half = reinterpret_cast<float2*>(tb + 138 * p + j);
#pragma unroll
      for (int tr = 0; tr < 2; ++tr) {
        float2 xv[16], rv[16];
#pragma unroll
        for (int n = 0; n < 16; ++n) {
          const unsigned wa = word_of(X[2 * tr + (n >> 3)], (n & 7) >> 1);
          const unsigned wb = word_of(X[4 + 2 * tr + (n >> 3)], (n & 7) >> 1);
          const float2 m = (n & 1) ? make_float2(i16_hi_m(wa), i16_hi_m(wb)) : make_float2(i16_lo_m(wa), i16_lo_m(wb));
          xv[n] = __fadd2_rn(m, make_float2(-8421376.0f, -8421376.0f));  // exact v
        }
        fwd16(xv, rv);
#pragma unroll
        for (int k = 0; k < 16; ++k) half[2 * (8 * k + (k >> 1)) + tr] = rv[k];
      }
    }
    __syncwarp();

    QuantTile fut;
    const bool have_fut = have_nxt && ok && c_t < t_stop;
    if (have_fut) {
      take(fut);
      ok = advance();
    }
    if (!kLevels) {
      if (have_fut) issue(fut, st);
      else cp_async_commit();
    }
    int16_t* const lvs = reinterpret_cast<int16_t*>(reinterpret_cast<uint4*>(tb + kZT2Units) + 256 * st);

    // ---- per column c = 2j + i: column pass (exact Y), quantise, error
    // energy, dequantise, inverse column pass, back into the same line
    float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int c = 2 * j + i;
      float4* const line = tb + 138 * p + 17 * j + 8 * i;
      float2 cv[16], y[16];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 v = line[q];
        cv[2 * q] = make_float2(v.x, v.y);
        cv[2 * q + 1] = make_float2(v.z, v.w);
      }
      fwd16(cv, y);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float k = kq[i][quant_uclass(u)], g = gq[i][quant_uclass(u)];
        // |Y| k as two scalar multiplies: the absolute value folds into them
        const float2 t = make_float2(__fmul_rn(fabsf(y[u].x), k), __fmul_rn(fabsf(y[u].y), k));
        const float2 b = __fadd2_rn(t, make_float2(0.5f, 0.5f));
        const float2 f = f2add_rm(b, make_float2(8388608.0f, 8388608.0f));  // floor(b) + 2^23
        const float2 L = __fadd2_rn(f, make_float2(-8388608.0f, -8388608.0f));
        // B - B' = Qstep (|Y| s / Qstep - L) ~ Qstep (t - L); Qstep^2 is applied per tile
        const float2 e = bsub(t, L);
        float2& sacc = (u & 1) ? acc1 : acc;
        sacc = __ffma2_rn(e, e, sacc);
        if (kLevels) {
          const int la = (int)(__float_as_uint(f.x) - 0x4B000000u), lb = (int)(__float_as_uint(f.y) - 0x4B000000u);
          const int hw = (kZigzag ? (int)((zzl[4 * i + (u >> 2)] >> (8 * (u & 3))) & 0xffu) : (16 * u + c)) ^ (16 * p);
          lvs[256 * p + hw] = (int16_t)(y[u].x < 0.f ? -la : la);
          lvs[256 * (p + 4) + hw] = (int16_t)(y[u].y < 0.f ? -lb : lb);
        }
        y[u] = f2copysign(__fmul2_rn(L, make_float2(g, g)), y[u]);
      }
      float2 uo[16];
      inv16(y, uo);
#pragma unroll
      for (int q = 0; q < 8; ++q) line[q] = make_float4(uo[2 * q].x, uo[2 * q].y, uo[2 * q + 1].x, uo[2 * q + 1].y);
    }
    __syncwarp();
    if (kLevels) {
      // the tile's levels, one 512-byte run per block, then refill the slot
      int16_t* const gl = levels + (cur.lvl - 256 * p);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        if (b >= cur.nb) break;
        const uint4 v = reinterpret_cast<const uint4*>(lvs + 256 * b)[lane ^ (2 * (b & 3))];
        __stcs(reinterpret_cast<uint4*>(gl + 256 * b + 8 * lane), v);
      }
      __syncwarp();
      if (have_fut) issue(fut, st);
      else cp_async_commit();
    }

    // ---- per row 2j + rr: gather (8-byte halves, conflict-free with the
    // row-order swap of the zonal kernel), inverse row pass, rint, pack, store
#pragma unroll
    for (int tr = 0; tr < 2; ++tr) {
      const int rr = tr ^ jb1;
      const float2* const fin = reinterpret_cast<const float2*>(tb + 138 * p + j) + rr;
      float2 v[16], z[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = fin[2 * (8 * c + (c >> 1))];
      inv16(v, z);
      unsigned oa[8], ob[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        // rint by the magic add 1.5 * 2^23 (|z| < 2^22), then saturate to int16
        const float2 m0 = __fadd2_rn(z[2 * n], make_float2(12582912.0f, 12582912.0f));
        const float2 m1 = __fadd2_rn(z[2 * n + 1], make_float2(12582912.0f, 12582912.0f));
        oa[n] = pack_s16((int)(__float_as_uint(m1.x) - 0x4B400000u), (int)(__float_as_uint(m0.x) - 0x4B400000u));
        ob[n] = pack_s16((int)(__float_as_uint(m1.y) - 0x4B400000u), (int)(__float_as_uint(m0.y) - 0x4B400000u));
      }
      uint8_t* d = cur.dst + rr * cur.dst_pitch;
      if (va) {
        __stcs(reinterpret_cast<uint4*>(d), make_uint4(oa[0], oa[1], oa[2], oa[3]));
        __stcs(reinterpret_cast<uint4*>(d + 16), make_uint4(oa[4], oa[5], oa[6], oa[7]));
      }
      if (vb) {
        __stcs(reinterpret_cast<uint4*>(d + 128), make_uint4(ob[0], ob[1], ob[2], ob[3]));
        __stcs(reinterpret_cast<uint4*>(d + 144), make_uint4(ob[4], ob[5], ob[6], ob[7]));
      }
    }

    acc = __fadd2_rn(acc, acc1);
    const float tot = warp_sum((va ? acc.x : 0.f) + (vb ? acc.y : 0.f));
    if (lane == 0) tile_sse[cur.t] = tot * qstep * qstep;
    __syncwarp();  // buffer reads done before the next tile's writes

    if (!have_nxt) break;
    cur = nxt;
    nxt = fut;
    have_nxt = have_fut;
    st ^= 1;
  }
  cp_async_wait<0>();
  if (!ok && lane == 0) set_status(status, kDevBadJob);
  pdl_launch_dependents();  // the PSNR finalize may now take this CTA's place
}

// --------------------------------------------------------------------------
// SSIM (Sec. 4, the measure of Wang et al. 2004): mean over the valid
// positions of the 11x11 Gaussian window (sigma 1.5) of
//   (2 mu_a mu_b + C1)(2 s_ab + C2) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 + s_b^2 + C2)).
// The window is separable: the 2-D normalised Gaussian is the outer product
// of the 1-D normalised one (kSsimW).  One CTA per tile of 20 x 128 window
// positions (65 KB of shared memory, three CTAs per SM), in two passes over
// the five moments of the centred pixels
// (a, b, a^2, b^2, ab with a = x - 128, which keeps the moment form
// E[xy] - E[x]E[y] well conditioned in FP32), (a, b) and (a^2, b^2) as
// packed pairs (one f32x2 instruction per pair):
//   input       the tile's 30 x 138 pixels of both images, copied to shared
//               memory with cp.async; the next tile's copy starts as soon as
//               the vertical pass has read this one;
//   vertical    thread c (< 138) walks column x0 + c down the 30 input rows
//               with 11 running sums per moment in registers (row r adds
//               w_k f(r) to output row r - k; output row r - 10 is then
//               complete), into the moment planes;
//   horizontal  a thread takes 8 consecutive positions of one row (lanes on
//               consecutive rows: odd 16-byte row strides keep the 16-byte
//               reads conflict-free) and finishes the 11 taps and the SSIM
//               value in registers.
// The tile's sum of SSIM values goes to tile_sum.
// --------------------------------------------------------------------------
constexpr int kSsimTR = kSsimTileRows, kSsimTC = kSsimTileCols;
constexpr int kSsimVC = kSsimTC + 10;   // columns of vertical moments
constexpr int kSsimIR = kSsimTR + 10;   // input rows of a tile
constexpr int kSsimIS = 144;            // bytes per staged input row (9 chunks of 16)
constexpr int kSsimVS2 = 142;           // row stride of a pair plane (float2): 71 chunks
constexpr int kSsimVS1 = 140;           // row stride of the ab plane (float): 35 chunks
constexpr int kSsimThreads = 160;
static_assert(kSsimTC == 128, "the horizontal pass is written for 128-column tiles");
__constant__ float kSsimW[11];

struct alignas(16) SsimSmem {
  float2 v2[2][kSsimTR][kSsimVS2];   // vertical (a, b) and (a^2, b^2)
  float v1[kSsimTR][kSsimVS1];       // vertical ab
  uint8_t in[2][kSsimIR][kSsimIS];   // input pixels of both images
  float red[kSsimThreads / 32];
};

struct SsimTile {
  const uint8_t* pa;
  const uint8_t* pb;
  long long ps, pd;
  int w, h, y0, x0;
  bool ok;
};

__device__ __forceinline__ SsimTile ssim_tile(const ImageJob* __restrict__ jobs, int njobs, long long t) {
  SsimTile T;
  int job = 0;
  find_job(jobs, njobs, t, job);
  const ImageJob* J = jobs + job;
  const long long tb = __ldg(&J->tile_begin);
  T.w = __ldg(&J->width);
  T.h = __ldg(&J->height);
  const int tiles_x = __ldg(&J->tiles_x);
  T.ok = t >= tb && t < tb + (long long)tiles_x * ((T.h - 10 + kSsimTR - 1) / kSsimTR) && tiles_x > 0;
  const int lt = T.ok ? (int)(t - tb) : 0, ty = lt / max(tiles_x, 1), tx = lt - ty * max(tiles_x, 1);
  T.y0 = ty * kSsimTR;
  T.x0 = tx * kSsimTC;
  T.pa = reinterpret_cast<const uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->src)));
  T.pb = reinterpret_cast<const uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->dst)));
  T.ps = __ldg(&J->src_pitch);
  T.pd = __ldg(&J->dst_pitch);
  return T;
}

// cp.async of a tile's input rows: 2 images x 30 rows x 9 chunks of 16 bytes;
// chunks past the image (width and pitch are multiples of 16) are zero-filled.
__device__ __forceinline__ void ssim_issue(SsimSmem& sm, const SsimTile& T, int tid) {
  for (int i = tid; i < 2 * kSsimIR * 9; i += kSsimThreads) {
    const int img = i / (kSsimIR * 9), rem = i - img * (kSsimIR * 9), r = rem / 9, k = rem - r * 9;
    const int y = T.y0 + r, x = T.x0 + 16 * k;
    const bool in = y < T.h && x < T.w;
    const uint8_t* g = img ? T.pb + (in ? y * T.pd + x : 0) : T.pa + (in ? y * T.ps + x : 0);
    cp_async16_zfill(&sm.in[img][r][16 * k], g, in ? 16 : 0);
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(kSsimThreads, 3)
ssim_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles, float* __restrict__ tile_sum,
            int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char ssmem[];
  SsimSmem& sm = *reinterpret_cast<SsimSmem*>(ssmem);
  const int tid = threadIdx.x;
  float wk[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) wk[k] = kSsimW[k];
  long long t = blockIdx.x;
  if (t >= ntiles) return;
  SsimTile T = ssim_tile(jobs, njobs, t);
  if (T.ok) ssim_issue(sm, T, tid);
  for (; t < ntiles; t += gridDim.x) {
    const long long tn = t + gridDim.x;
    cp_async_wait<0>();
    __syncthreads();  // this tile's input is in; the previous tile's moment reads are done
    if (T.ok && tid < kSsimVC) {
      float2 acc2[11][2];
      float acc1[11];
#pragma unroll
      for (int s = 0; s < 11; ++s) {
        acc2[s][0] = acc2[s][1] = make_float2(0.f, 0.f);
        acc1[s] = 0.f;
      }
#pragma unroll
      for (int r = 0; r < kSsimIR; ++r) {
        const float a = (float)sm.in[0][r][tid] - 128.f, b = (float)sm.in[1][r][tid] - 128.f;
        const float2 ab = make_float2(a, b), sq = __fmul2_rn(ab, ab);
        const float x = a * b;
#pragma unroll
        for (int k = 0; k < 11; ++k) {
          const int sl = (r - k + 22) % 11;  // slot of output row r - k
          const float2 wk2 = make_float2(wk[k], wk[k]);
          acc2[sl][0] = __ffma2_rn(wk2, ab, acc2[sl][0]);
          acc2[sl][1] = __ffma2_rn(wk2, sq, acc2[sl][1]);
          acc1[sl] = fmaf(wk[k], x, acc1[sl]);
        }
        const int o = r - 10, sl = (r + 1) % 11;  // output row r - 10 is complete
        if (o >= 0) {
          sm.v2[0][o][tid] = acc2[sl][0];
          sm.v2[1][o][tid] = acc2[sl][1];
          sm.v1[o][tid] = acc1[sl];
        }
        acc2[sl][0] = acc2[sl][1] = make_float2(0.f, 0.f);
        acc1[sl] = 0.f;
      }
    }
    __syncthreads();  // moments complete; the input buffer is free
    const SsimTile cur = T;
    if (tn < ntiles) {
      T = ssim_tile(jobs, njobs, tn);
      if (T.ok) ssim_issue(sm, T, tid);
    }
    if (!cur.ok) {
      if (tid == 0) {
        set_status(status, kDevBadJob);
        tile_sum[t] = 0.f;
      }
      continue;
    }
    const int mh = cur.h - 10, mw = cur.w - 10;
    float part = 0.f;
    for (int i = tid; i < kSsimTR * (kSsimTC / 8); i += kSsimThreads) {
      const int g = i / kSsimTR, row = i - g * kSsimTR, c0 = 8 * g;
      float2 m2[2][8];
      float m1[8];
#pragma unroll
      for (int pl = 0; pl < 2; ++pl) {
        float2 in[18];
        const float4* src = reinterpret_cast<const float4*>(&sm.v2[pl][row][c0]);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const float4 v = src[q];
          in[2 * q] = make_float2(v.x, v.y);
          in[2 * q + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int k = 0; k < 11; ++k) s2 = __ffma2_rn(make_float2(wk[k], wk[k]), in[o + k], s2);
          m2[pl][o] = s2;
        }
      }
      {
        float in[20];
        const float4* src = reinterpret_cast<const float4*>(&sm.v1[row][c0]);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const float4 v = src[q];
          in[4 * q] = v.x;
          in[4 * q + 1] = v.y;
          in[4 * q + 2] = v.z;
          in[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          float s1 = 0.f;
#pragma unroll
          for (int k = 0; k < 11; ++k) s1 = fmaf(wk[k], in[o + k], s1);
          m1[o] = s1;
        }
      }
      const bool rin = cur.y0 + row < mh;
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        // back from the centred values: mu = mu' + 128; variances and covariance unchanged
        const float2 mu = m2[0][o], ex2 = m2[1][o];
        const float ma = mu.x + 128.f, mb = mu.y + 128.f;
        const float saa = ex2.x - mu.x * mu.x, sbb = ex2.y - mu.y * mu.y, sab = m1[o] - mu.x * mu.y;
        const float c1 = 6.5025f, c2 = 58.5225f;  // (0.01 * 255)^2, (0.03 * 255)^2
        const float v = __fdividef((2.f * ma * mb + c1) * (2.f * sab + c2), (ma * ma + mb * mb + c1) * (saa + sbb + c2));
        if (rin && cur.x0 + c0 + o < mw) part += v;
      }
    }
    part = warp_sum(part);
    if ((tid & 31) == 0) sm.red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < kSsimThreads / 32; ++k) s += sm.red[k];
      tile_sum[t] = s;
    }
  }
  cp_async_wait<0>();
}

// MSSIM per image: the tile sums in a fixed order (FP64) over the number of
// window positions.
__global__ void ssim_finalize_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles,
                                     const float* __restrict__ tile_sum, double* __restrict__ out) {
  pdl_wait_primary();
  const int lane = threadIdx.x & 31;
  const int job = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (job >= njobs) return;
  const long long b = jobs[job].tile_begin;
  const long long e = (job + 1 < njobs) ? jobs[job + 1].tile_begin : ntiles;
  double s = 0.0;
  for (long long t = b + lane; t < e; t += 32) s += (double)tile_sum[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[job] = s / ((double)(jobs[job].width - 10) * (double)(jobs[job].height - 10));
}

// --------------------------------------------------------------------------
// Exact-DCT baseline of the zonal path: the same Sec. 4 procedure with the
// orthonormal 16-point DCT-II matrix C (Sec. 3.2) in place of C_hat, as
// dense FP32 products (16 multiply-adds per output), for comparison with
// the multiplierless transform.  Per block: B = C A C^T, keep the first r
// zig-zag coefficients, A' = C^T B' C, rint (ties to even) and clamp to
// 0..255; the dropped energy is the SSE of the unrounded reconstruction
// (C is orthonormal).  Same tiling, staging and in-place line-per-column
// transpose as the quantisation kernel.
// --------------------------------------------------------------------------
__constant__ float kDctC[16][16];  // C[k][j], FP32 of the FP64 values

// Row k of C, broadcast to both halves of a pair (the loops over k stay
// rolled: k is warp-uniform, so C[k][.] comes through the uniform path and
// no per-thread array is indexed at run time).
__device__ __forceinline__ float2 dct_c2(int k, int jj) { return make_float2(kDctC[k][jj], kDctC[k][jj]); }

constexpr int kDStageUnits = 2 * 4 * 32;
constexpr int kDctWarpSmemBytes = 16 * (kZT2Units + kDStageUnits);

__global__ void __launch_bounds__(128, 3)
dct_zonal_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles_ll,
                 const float2* __restrict__ wtab, float* __restrict__ tile_sse, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char dsmem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane & 3, j = lane >> 2, jb1 = (j >> 1) & 1;
  float4* const tb = reinterpret_cast<float4*>(dsmem + warp * kDctWarpSmemBytes);
  uint4* const stg = reinterpret_cast<uint4*>(tb + kZT2Units) + lane;  // + 128 s + 32 k
  const int ntiles = (int)ntiles_ll;
  constexpr int kWarps = 4;
  const int nwarps = gridDim.x * kWarps;
  const int per_warp = (ntiles + nwarps - 1) / nwarps;
  const int t_first = (blockIdx.x * kWarps + warp) * per_warp;
  const int t_stop = min(ntiles, t_first + per_warp);
  if (t_first >= t_stop) return;

  int c_t = 0, c_end = 0, tiles_x = 1, tx = 0, nb_last = 8, r_job = 0, src_pitch = 0, dst_pitch = 0;
  const uint8_t* src_band = nullptr;
  uint8_t* dst_band = nullptr;
  auto enter = [&](int t) -> bool {
    int job;
    find_job(jobs, njobs, t, job);
    const ImageJob* J = jobs + job;
    const long long tb0 = __ldg(&J->tile_begin);
    tiles_x = __ldg(&J->tiles_x);
    const long long te = tb0 + (long long)tiles_x * (__ldg(&J->height) >> 4);
    if (t < tb0 || t >= te || tiles_x < 1) return false;
    c_end = (int)min(te, (long long)t_stop);
    const int lt = (int)(t - tb0);
    const int ty = lt / tiles_x;
    tx = lt - ty * tiles_x;
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
  auto take = [&](ZonalTile& z) {
    z.src = src_band + tx * kTileW;
    z.dst = dst_band + tx * kTileW;
    z.src_pitch = src_pitch;
    z.dst_pitch = dst_pitch;
    z.nb = tx == tiles_x - 1 ? nb_last : 8;
    z.t = c_t;
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
  auto issue = [&](const ZonalTile& z, int st) {
    uint4* d = stg + 128 * st;
    if (p < z.nb) {
      cp_async16(d, z.src);
      cp_async16(d + 32, z.src + z.src_pitch);
    }
    if (p + 4 < z.nb) {
      cp_async16(d + 64, z.src + 64);
      cp_async16(d + 96, z.src + 64 + z.src_pitch);
    }
    cp_async_commit();
  };

  if (!enter(t_first)) {
    if (lane == 0) set_status(status, kDevBadJob);
    return;
  }
  bool ok = true;
  int wr = -1;
  unsigned keep = 0;  // bit 16 i + u: coefficient (u, column 2j + i) is kept
  ZonalTile cur, nxt;
  take(cur);
  ok = advance();
  issue(cur, 0);
  bool have_nxt = ok && c_t < t_stop;
  if (have_nxt) {
    take(nxt);
    ok = advance();
    issue(nxt, 1);
  } else {
    cp_async_commit();
  }
  int st = 0;
  while (true) {
    cp_async_wait<1>();
    if (cur.r != wr) {  // the zig-zag mask of r from the zonal table (kept <=> weight != 0)
      keep = 0;
      const float2* w = wtab + (long long)cur.r * 256;
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (__ldg(w + (2 * j + i) * 16 + u).x != 0.f) keep |= 1u << (16 * i + u);
      wr = cur.r;
    }
    uint4 X[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) X[k] = stg[128 * st + 32 * k];
    const bool va = p < cur.nb, vb = p + 4 < cur.nb;

    // ---- row pass: 2^23 + x by a byte permute, minus 2^23, then C
    {
      float2* const half = reinterpret_cast<float2*>(tb + 138 * p + j);
#pragma unroll
      for (int tr = 0; tr < 2; ++tr) {
        float2 xv[16];
#pragma unroll
        for (int n = 0; n < 16; ++n) {
          const float2 m = make_float2(__uint_as_float(__byte_perm(word_of(X[tr], n >> 2), 0x4B000000u, 0x7440u | (n & 3))),
                                       __uint_as_float(__byte_perm(word_of(X[2 + tr], n >> 2), 0x4B000000u, 0x7440u | (n & 3))));
          xv[n] = __fadd2_rn(m, make_float2(-8388608.0f, -8388608.0f));
        }
#pragma unroll 1
        for (int k = 0; k < 16; ++k) {
          float2 y = make_float2(0.f, 0.f);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) y = __ffma2_rn(dct_c2(k, jj), xv[jj], y);
          half[2 * (8 * k + (k >> 1)) + tr] = y;
        }
      }
    }
    __syncwarp();

    ZonalTile fut;
    const bool have_fut = have_nxt && ok && c_t < t_stop;
    if (have_fut) {
      take(fut);
      ok = advance();
      issue(fut, st);
    } else {
      cp_async_commit();
    }

    // ---- columns: C, mask, dropped energy, C^T, in place
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float4* const line = tb + 138 * p + 17 * j + 8 * i;
      float2 cv[16], uo[16];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 v = line[q];
        cv[2 * q] = make_float2(v.x, v.y);
        cv[2 * q + 1] = make_float2(v.z, v.w);
        uo[2 * q] = uo[2 * q + 1] = make_float2(0.f, 0.f);
      }
      // per coefficient u: B(u) = C(u, :) . column, the mask, then its
      // contribution C(u, m) B'(u) to every output m (outer-product form)
#pragma unroll 1
      for (int u = 0; u < 16; ++u) {
        float2 y = make_float2(0.f, 0.f);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) y = __ffma2_rn(dct_c2(u, jj), cv[jj], y);
        if (!((keep >> (16 * i + u)) & 1u)) {
          acc = __ffma2_rn(y, y, acc);
          y = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < 16; ++m) uo[m] = __ffma2_rn(dct_c2(u, m), y, uo[m]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) line[q] = make_float4(uo[2 * q].x, uo[2 * q].y, uo[2 * q + 1].x, uo[2 * q + 1].y);
    }
    __syncwarp();

    // ---- rows: C^T, rint, clamp, pack, store
#pragma unroll
    for (int tr = 0; tr < 2; ++tr) {
      const int rr = tr ^ jb1;
      const float2* const fin = reinterpret_cast<const float2*>(tb + 138 * p + j) + rr;
      float2 z[16];
#pragma unroll
      for (int n = 0; n < 16; ++n) z[n] = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int c = 0; c < 16; ++c) {
        const float2 v = fin[2 * (8 * c + (c >> 1))];
#pragma unroll
        for (int n = 0; n < 16; ++n) z[n] = __ffma2_rn(dct_c2(c, n), v, z[n]);
      }
      unsigned oa[4], ob[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        int qa[4], qb[4];
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
          // rint by the magic add 1.5 * 2^23, then the saturating u8 pack
          const float2 m = __fadd2_rn(z[4 * g + e4], make_float2(12582912.0f, 12582912.0f));
          qa[e4] = (int)(__float_as_uint(m.x) - 0x4B400000u);
          qb[e4] = (int)(__float_as_uint(m.y) - 0x4B400000u);
        }
        oa[g] = pack_u8(qa[1], qa[0], pack_u8(qa[3], qa[2], 0u));
        ob[g] = pack_u8(qb[1], qb[0], pack_u8(qb[3], qb[2], 0u));
      }
      uint8_t* d = cur.dst + rr * cur.dst_pitch;
      if (va) __stcs(reinterpret_cast<uint4*>(d), make_uint4(oa[0], oa[1], oa[2], oa[3]));
      if (vb) __stcs(reinterpret_cast<uint4*>(d + 64), make_uint4(ob[0], ob[1], ob[2], ob[3]));
    }

    const float tot = warp_sum((va ? acc.x : 0.f) + (vb ? acc.y : 0.f));
    if (lane == 0) tile_sse[cur.t] = tot;
    __syncwarp();

    if (!have_nxt) break;
    cur = nxt;
    nxt = fut;
    have_nxt = have_fut;
    st ^= 1;
  }
  cp_async_wait<0>();
  if (!ok && lane == 0) set_status(status, kDevBadJob);
  pdl_launch_dependents();  // the PSNR finalize may now take this CTA's place
}

// --------------------------------------------------------------------------
// Per-image PSNR from the per-tile SSE partials (FP64, fixed summation order).
//
// The kernel sits between two launches of the fused kernel, so its length is
// the length of its longest dependent chain, and FP64 operations are slow on
// this part.  The logarithm is therefore split: for a normal double
// x = m 2^e (1 <= m < 2, taken exactly from the bit pattern) log10 x =
// e log10 2 + log10 m, with log10 m evaluated in FP32 (absolute error below
// 1e-7, i.e. below 1e-6 dB of PSNR), and PSNR = 10 (log10(peak^2 N) - log10 SSE)
// needs no FP64 division.
// --------------------------------------------------------------------------
__device__ __forceinline__ double log10_split(double x) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff) return log10(x);  // zero, subnormal, inf, nan
  const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  return (double)(ex - 1023) * 0.301029995663981195 + (double)log10f((float)m);
}

__global__ void psnr_finalize_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles,
                                     const float* __restrict__ tile_sse, double peak,
                                     double* __restrict__ psnr, double* __restrict__ sse_out) {
  const int lane = threadIdx.x & 31;
  const int job = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  // the job table is not written by the producing kernel: read it before the wait
  long long b = 0, e = 0;
  double lpeak = 0.0;  // log10(peak^2 N)
  if (job < njobs) {
    b = jobs[job].tile_begin;
    e = (job + 1 < njobs) ? jobs[job + 1].tile_begin : ntiles;
    lpeak = log10_split(peak * peak * ((double)jobs[job].width * (double)jobs[job].height));
  }
  pdl_wait_primary();  // the producing kernel's partials are complete and visible
  if (job >= njobs) return;
  double s = 0.0;
  long long t = b + lane;
  for (; t + 96 < e; t += 128) {  // four loads in flight, same order of additions
    const float a0 = tile_sse[t], a1 = tile_sse[t + 32], a2 = tile_sse[t + 64], a3 = tile_sse[t + 96];
    s += (double)a0;
    s += (double)a1;
    s += (double)a2;
    s += (double)a3;
  }
  for (; t < e; t += 32) s += (double)tile_sse[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    psnr[job] = s > 0.0 ? 10.0 * (lpeak - log10_split(s)) : CUDART_INF;
    if (sse_out) sse_out[job] = s;
  }
}

// --------------------------------------------------------------------------
// PSNR of two images, exact integer SSE accumulated in the output slot.
// --------------------------------------------------------------------------
template <int kDtype>
__global__ void psnr_pair_kernel(const uint8_t* __restrict__ a, long long pa, const uint8_t* __restrict__ b,
                                 long long pb, int w, int h, unsigned long long* __restrict__ acc) {
  unsigned long long s = 0;
  const long long n = (long long)w * h;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long y = i / w, x = i - y * w;
    long long d;
    if (kDtype == 0) d = (long long)a[y * pa + x] - (long long)b[y * pb + x];
    else d = (long long)reinterpret_cast<const int16_t*>(a + y * pa)[x] - (long long)reinterpret_cast<const int16_t*>(b + y * pb)[x];
    s += (unsigned long long)(d * d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(acc, s);
}

__global__ void psnr_pair_finish(unsigned long long* slot, double npx, double peak) {
  const unsigned long long s = *slot;
  *reinterpret_cast<double*>(slot) = s ? 10.0 * log10(peak * peak * npx / (double)s) : CUDART_INF;
}

// --------------------------------------------------------------------------
// Launchers
// --------------------------------------------------------------------------
template <class K, class... Args>
static cudaError_t launch_with_smem(K kernel, int grid, int threads, int smem, cudaStream_t stream, Args... args) {
  // dynamic shared memory above 48 KB must be enabled per device
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  kernel<<<grid, threads, smem, stream>>>(args...);
  return cudaGetLastError();
}


template <class K>
static cudaError_t occupancy_with_smem(int* n, K kernel, int threads, int smem) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kernel, threads, smem);
}

static int config_index(const ZonalConfig& c) {
  if (!c.prefetch || c.warps != 4) return -1;
  return c.variant == kZonalSwar ? 0
         : c.variant == kZonalF32 ? 1
         : c.variant == kZonalMma ? 2
         : c.variant == kZonalTc  ? 3
                                  : -1;
}

bool zonal_config_supported(const ZonalConfig& c) { return config_index(c) >= 0; }

cudaError_t launch_zonal_config(const ZonalConfig& cfg, const ImageJob* d_jobs, int njobs, long long ntiles,
                                const float2* d_wtab, float* d_tile_sse, int* d_status, int grid,
                                cudaStream_t stream, bool dependent, bool early) {
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles >= (1LL << 30)) return cudaErrorInvalidValue;  // tile indices are 32-bit in the kernels
  const int threads = 32 * cfg.warps;
  const int pe = early ? 1 : 0;
  switch (config_index(cfg)) {
    case 0:
      return launch_chained(zonal_f32_kernel<4, true>, grid, threads, 4 * kZonalWarpSmemBytes, stream, dependent,
                            d_jobs, njobs, ntiles, d_wtab, d_tile_sse, d_status, pe);
    case 1:
      return launch_chained(zonal_f32_kernel<4, false>, grid, threads, 4 * kZonalWarpSmemBytes, stream, dependent,
                            d_jobs, njobs, ntiles, d_wtab, d_tile_sse, d_status, pe);
    case 2:
      return launch_chained(zonal_mma_kernel<4>, grid, threads, 4 * kZonalMmaWarpSmemBytes, stream, dependent,
                            d_jobs, njobs, ntiles, d_wtab, d_tile_sse, d_status, pe);
    case 3:
      return launch_zonal_tc(d_jobs, njobs, ntiles, d_wtab, d_tile_sse, d_status, grid, stream, dependent, early,
                             cfg.test_stall != 0);
  }
  return cudaErrorInvalidValue;
}

int zonal_config_max_ctas_per_sm(const ZonalConfig& cfg) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const int zs = kZonalWarpSmemBytes;
  switch (config_index(cfg)) {
    case 0: e = occupancy_with_smem(&n, zonal_f32_kernel<4, true>, 128, 4 * zs); break;
    case 1: e = occupancy_with_smem(&n, zonal_f32_kernel<4, false>, 128, 4 * zs); break;
    case 2: e = occupancy_with_smem(&n, zonal_mma_kernel<4>, 128, 4 * kZonalMmaWarpSmemBytes); break;
    case 3: return zonal_tc_max_ctas_per_sm();
  }
  return (e == cudaSuccess && n > 0) ? n : 1;
}

ZonalConfig default_zonal_config() { return ZonalConfig{kZonalSwar, kZonalWarps, 1}; }

cudaError_t launch_quant(const ImageJob* d_jobs, int njobs, long long ntiles, const float4* d_qtab,
                         int16_t* d_levels, bool zigzag, float* d_tile_sse, int* d_status, int grid,
                         cudaStream_t stream) {
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles >= (1LL << 30)) return cudaErrorInvalidValue;  // tile indices are 32-bit in the kernel
  if (d_levels && zigzag)
    return launch_with_smem(quant_kernel<true, true>, grid, 128, 4 * kQuantWarpSmemBytes, stream, d_jobs, njobs,
                            ntiles, d_qtab, d_levels, d_tile_sse, d_status);
  if (d_levels)
    return launch_with_smem(quant_kernel<true, false>, grid, 128, 4 * kQuantWarpSmemBytes, stream, d_jobs, njobs,
                            ntiles, d_qtab, d_levels, d_tile_sse, d_status);
  return launch_with_smem(quant_kernel<false, false>, grid, 128, 4 * kQuantWarpSmemBytes, stream, d_jobs, njobs,
                          ntiles, d_qtab, d_levels, d_tile_sse, d_status);
}

cudaError_t launch_psnr_finalize(const ImageJob* d_jobs, int njobs, long long ntiles, const float* d_tile_sse,
                                 double peak, double* d_psnr, double* d_sse, cudaStream_t stream) {
  if (njobs <= 0) return cudaSuccess;
  const int warps = 8;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((njobs + warps - 1) / warps);
  cfg.blockDim = dim3(32 * warps);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, psnr_finalize_kernel, d_jobs, njobs, ntiles, d_tile_sse, peak, d_psnr, d_sse);
}

cudaError_t launch_psnr_pair(int dtype, const void* d_a, long long pitch_a, const void* d_b, long long pitch_b,
                             int w, int h, double* d_out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double), stream);
  if (e != cudaSuccess) return e;
  unsigned long long* slot = reinterpret_cast<unsigned long long*>(d_out);
  const long long n = (long long)w * h;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (dtype == 0)
    psnr_pair_kernel<0><<<grid, 256, 0, stream>>>((const uint8_t*)d_a, pitch_a, (const uint8_t*)d_b, pitch_b, w, h, slot);
  else
    psnr_pair_kernel<1><<<grid, 256, 0, stream>>>((const uint8_t*)d_a, pitch_a, (const uint8_t*)d_b, pitch_b, w, h, slot);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  psnr_pair_finish<<<1, 1, 0, stream>>>(slot, (double)n, 255.0);
  return cudaGetLastError();
}

int zonal_ctas_per_sm() { return zonal_config_max_ctas_per_sm(default_zonal_config()); }
cudaError_t launch_ssim(const ImageJob* d_jobs, int njobs, long long ntiles, float* d_tile_sum, double* d_out,
                        int* d_status, int num_sms, cudaStream_t stream) {
  if (ntiles <= 0 || njobs <= 0) return cudaSuccess;
  static std::atomic<bool> weights_ready[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !weights_ready[dev].load()) {
    // the 1-D normalised Gaussian of standard deviation 1.5 on -5 .. 5
    double g[11], sum = 0.0;
    for (int k = 0; k < 11; ++k) sum += (g[k] = std::exp(-(k - 5.0) * (k - 5.0) / 4.5));
    float w[11];
    for (int k = 0; k < 11; ++k) w[k] = (float)(g[k] / sum);
    e = cudaMemcpyToSymbolAsync(kSsimW, w, sizeof(w), 0, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    if (dev < 64) weights_ready[dev].store(true);
  }
  const int smem = (int)sizeof(SsimSmem);
  int per_sm = 0;
  e = occupancy_with_smem(&per_sm, ssim_kernel, kSsimThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(ntiles, (long long)num_sms * std::max(1, per_sm));
  e = launch_with_smem(ssim_kernel, grid, kSsimThreads, smem, stream, d_jobs, njobs, ntiles, d_tile_sum, d_status);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((njobs + 7) / 8);
  cfg.blockDim = dim3(256);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ssim_finalize_kernel, d_jobs, njobs, ntiles, (const float*)d_tile_sum, d_out);
}

cudaError_t launch_zonal_dct(const ImageJob* d_jobs, int njobs, long long ntiles, const float2* d_wtab,
                             float* d_tile_sse, int* d_status, int num_sms, cudaStream_t stream) {
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles >= (1LL << 30)) return cudaErrorInvalidValue;
  static std::atomic<bool> ready[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !ready[dev].load()) {
    // the orthonormal DCT-II matrix, FP64 -> FP32
    float c[16][16];
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < 16; ++k)
      for (int jj = 0; jj < 16; ++jj)
        c[k][jj] = (float)((k == 0 ? std::sqrt(1.0 / 16.0) : std::sqrt(2.0 / 16.0)) *
                           std::cos(pi * (2 * jj + 1) * k / 32.0));
    e = cudaMemcpyToSymbolAsync(kDctC, c, sizeof(c), 0, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    if (dev < 64) ready[dev].store(true);
  }
  int per_sm = 0;
  e = occupancy_with_smem(&per_sm, dct_zonal_kernel, 128, 4 * kDctWarpSmemBytes);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>((long long)num_sms * std::max(1, per_sm), (ntiles + 3) / 4);
  return launch_with_smem(dct_zonal_kernel, grid, 128, 4 * kDctWarpSmemBytes, stream, d_jobs, njobs, ntiles, d_wtab,
                          d_tile_sse, d_status);
}

int quant_ctas_per_sm() {
  int n = 0;
  if (occupancy_with_smem(&n, quant_kernel<false, false>, 128, 4 * kQuantWarpSmemBytes) != cudaSuccess || n < 1) n = 1;
  return n;
}

}  // namespace atdct16
