// Fused zonal compression (the Sec. 4 procedure: forward 2-D transform, keep
// the first r zig-zag coefficients, S^2 scaling, exact inverse, round, PSNR
// partials) with both forward passes on the fifth-generation tensor cores.
//
// The forward transform Y = T X T^T of a block is two exact 16 x 16 integer
// products, and tcgen05.mma runs each of them for 128 block rows (or
// columns) of two blocks at a time: M = 128, N = 32, K = 32 (two K = 16
// instructions) f16 products with f32 accumulators in tensor memory (TMEM).
// Row L of an operand carries a pair of blocks (p, p + 4) side by side in K,
// and B is block-diagonal with its columns interleaved, so that the
// accumulator's column 2 c + h belongs to block p + 4 h: one TMEM load then
// hands each thread its values as ready-made (block p, block p + 4) pairs.
//   pass 1  A1[(tile, p, m), 16 h + n] = 1024 + x_{p+4h}[m][n] (one byte
//           permute makes two f16 from two pixels), B1[16 h + n][2 v + h] =
//           T[v][n]: P = A1 B1 holds 1024 sum_n T[v][n] + (T x) per block
//           row; only v = 0 carries the 16384, and P[.][0] - 18432 =
//           sum_n (x - 128) centres it, so every entry of P lies in
//           [-2048, 2040] and is exact in f16;
//   pass 2  A2[(tile, p, v), 16 h + m] = P_{p+4h}[m][v] written MN-major
//           (the thread holding row m of P writes it as column m of A2, so
//           the transposition between the passes costs nothing),
//           B2[16 h + m][2 u + h] = 256 T[u][m]: the accumulator holds
//           256 Y_c, Y_c the coefficients of the block centred at 128
//           (|256 Y_c| <= 2^23, exact in f32); adding 2^23 at (0, 0) gives
//           256 Y.
// All products and partial sums are integers below 2^24, so both passes are
// exact.  The rest (mask and S^2 weights as W_u W_v / 256 per coefficient,
// dropped energy, inverse column pass, a warp-private back-transpose, inverse
// row pass, exact rounding of Z / 2304, u8 stores) is the general kernel's
// FP32 arithmetic on packed pairs (blocks p, p + 4).
//
// Work decomposition.  A CTA is one warpgroup (4 warps) and walks a
// contiguous range of tiles (16 x 128 pixels, 8 blocks) two at a time.  The
// thread with TMEM lane L = 64 tau + 16 p + i (warp L >> 5) owns, in tile tau
// of the pair, row i of blocks p and p + 4 on the pixel side and column v = i
// of the same blocks on the coefficient side.
// Software pipeline, per pair k:
//   wait MMA2(k); wait MMA1(k+1); P(k+1) -> A2; staged pixels of k+2 -> A1;
//   copy the rows of k+3 into the staging slot; Y(k) -> registers; one CTA
//   barrier; thread 0 issues MMA2(k+1) and MMA1(k+2); then the CUDA-core work
//   of pair k runs while the tensor core computes the next products.  Each
//   warp keeps the output row, pitch, tile index, r and block count of its
//   tiles in flight in a four-entry ring in shared memory, and its tile's
//   S^2 weights in a padded shared copy refreshed when r changes.
// Every wait on the tensor core is bounded (the kernel then records a device
// timeout, stops issuing, frees its TMEM and returns).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "atdct16_butterfly.cuh"
#include "atdct16_device.cuh"
#include "atdct16_internal.h"
#include "atdct16_tc.cuh"

namespace atdct16 {

namespace {

// Shared memory of one CTA (bytes).  Operand layouts (no swizzle): SBO 512
// between 8-groups along M or N, LBO 128 between 8-groups along K.
constexpr int kTcA1 = 0;          // pass-1 operand: 128 x 32 f16, K-major
constexpr int kTcA2 = 8192;       // pass-2 operand: 128 x 32 f16, MN-major
constexpr int kTcB = 16384;       // B1 and B2: 32 x 32 f16, K-major, 2048 each
constexpr int kTcStage = 20480;   // input rows: 2 slots x (block p, block p + 4) x 128 threads x 16 bytes
constexpr int kTcTr = 28672;      // back-transpose: per warp 2 x 16 x 18 float2 (4608 bytes)
constexpr int kTcRing = 47104;    // per warp 4 x 32 bytes: the tiles of the pairs in flight
constexpr int kTcPart = 47616;    // tile-energy partials of the second warp of each tile, [2 slots][2 tiles]
constexpr int kTcBar = 47632;     // mbarriers: MMA1 and MMA2 completion
constexpr int kTcSlot = 47648;    // the TMEM address written by tcgen05.alloc
constexpr int kTcW = 47664;       // per warp: its tile's weights, 16 columns at 9-unit strides (2304 bytes)
constexpr int kTcSmemBytes = 56880;
constexpr unsigned kTcCols = 64;  // TMEM columns: P (32 f32), Y (32 f32)
constexpr long long kTcWaitCycles = 1LL << 30;  // about 0.5 s per wait on the tensor core

// (lo, hi) -> f16x2 with lo in the low half (exact for the integers used)
__device__ __forceinline__ unsigned f16x2(float lo, float hi) {
  unsigned d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// The 16 pixels of one block row as f16 1024 + x, K = 8 g .. 8 g + 7 at a +
// 128 g (g = 0, 1) of the K-major pass-1 operand.
__device__ __forceinline__ void store_row_f16(unsigned char* a, const uint4& x) {
  const unsigned h = 0x64646464u;  // the high byte of the f16 1024 + x, x < 256
  *reinterpret_cast<uint4*>(a) = make_uint4(__byte_perm(x.x, h, 0x4140u), __byte_perm(x.x, h, 0x4342u),
                                            __byte_perm(x.y, h, 0x4140u), __byte_perm(x.y, h, 0x4342u));
  *reinterpret_cast<uint4*>(a + 128) = make_uint4(__byte_perm(x.z, h, 0x4140u), __byte_perm(x.z, h, 0x4342u),
                                                  __byte_perm(x.w, h, 0x4140u), __byte_perm(x.w, h, 0x4342u));
}

}  // namespace

__global__ void __launch_bounds__(128, 4)
zonal_tc_kernel(const ImageJob* __restrict__ jobs, int njobs, long long ntiles_ll, const float2* __restrict__ wtab,
                float* __restrict__ tile_sse, int* __restrict__ status, int pdl_early, int stall) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tau = warp >> 1;                   // tile of the pair
  const int p = 2 * (warp & 1) + (lane >> 4);  // block pair (p, p + 4)
  const int i16 = lane & 15;                   // pixel row m / coefficient column v
  const int ntiles = (int)ntiles_ll;           // the launcher checks ntiles < 2^30

  // the CTA's contiguous tile range, an even count except at the end
  const int per_cta = 2 * ((ntiles + 2 * (int)gridDim.x - 1) / (2 * (int)gridDim.x));
  const int c_first = blockIdx.x * per_cta;
  const int c_stop = min(ntiles, c_first + per_cta);
  if (pdl_early) pdl_launch_dependents();  // the next class's kernel may be scheduled
  if (c_first >= c_stop) {
    pdl_chain_exit();
    return;
  }
  const int npairs = (c_stop - c_first + 1) >> 1;

  unsigned* const tslot = reinterpret_cast<unsigned*>(tsm + kTcSlot);
  const unsigned bar1 = tc::smem_u32(tsm + kTcBar), bar2 = bar1 + 8;
  float* const part = reinterpret_cast<float*>(tsm + kTcPart);
  uint4* const ring = reinterpret_cast<uint4*>(tsm + kTcRing) + 8 * warp;  // entry e: units 2 e, 2 e + 1

  // ---- set-up: TMEM, mbarriers, the constant B operands
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tslot), kTcCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar1, 1);
    tc::mbar_init(bar2, 1);
    tc::fence_mbar_init();
  }
  if (tid < 16) {  // column n = tid of T (the butterfly's response to a unit vector) into both B
    int e[16], col[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) e[k] = k == tid ? 1 : 0;
    fwd16(e, col);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 16 * h + tid;
#pragma unroll
      for (int v = 0; v < 16; ++v) {
        const unsigned short one = col[v] == 0 ? 0 : (col[v] > 0 ? 0x3C00 : 0xBC00);  // f16 0, 1, -1
        const unsigned short w256 = col[v] == 0 ? 0 : (col[v] > 0 ? 0x5C00 : 0xDC00);  // f16 0, 256, -256
        const int n = 2 * v + h, nz = 2 * v + 1 - h;  // the entry and its zero partner in row k
        const int off = (n & 7) * 16 + (k & 7) * 2 + (n >> 3) * 512 + (k >> 3) * 128;
        const int offz = (nz & 7) * 16 + (k & 7) * 2 + (nz >> 3) * 512 + (k >> 3) * 128;
        *reinterpret_cast<unsigned short*>(tsm + kTcB + off) = one;
        *reinterpret_cast<unsigned short*>(tsm + kTcB + 2048 + off) = w256;
        *reinterpret_cast<unsigned short*>(tsm + kTcB + offz) = 0;
        *reinterpret_cast<unsigned short*>(tsm + kTcB + 2048 + offz) = 0;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const unsigned tbase = *tslot;
  const unsigned tlane = tbase + ((unsigned)(32 * warp) << 16);  // this warp's TMEM lanes
  const unsigned idK = tc::idesc_f16_f32(128, 32, false, false), idMN = tc::idesc_f16_f32(128, 32, true, false);
  const unsigned long long dA1 = tc::smem_desc(tc::smem_u32(tsm + kTcA1), 128, 512);
  const unsigned long long dA2 = tc::smem_desc(tc::smem_u32(tsm + kTcA2), 128, 512);
  const unsigned long long dB1 = tc::smem_desc(tc::smem_u32(tsm + kTcB), 128, 512);
  const unsigned long long dB2 = tc::smem_desc(tc::smem_u32(tsm + kTcB + 2048), 128, 512);
  constexpr unsigned long long kK16 = 256 >> 4;  // the second K half: two 8-groups (2 x LBO) on

  // ---- the warp's tile cursor over tiles c_first + tau + 2 k
  const int t_stop = c_stop;
  int c_t = 0, c_end = 0, tiles_x = 1, tx = 0, nb_last = 8, r_job = 0, src_pitch = 0, dst_pitch = 0, t_shift = 0;
  const uint8_t* src_band = nullptr;  // row i16 of block p in tile column 0 of the band
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
    const long long row = (long long)ty * kTileH + i16;
    src_band = reinterpret_cast<const uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->src))) +
               row * src_pitch + 16 * p;
    dst_band = reinterpret_cast<uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->dst))) +
               row * dst_pitch + 16 * p;
    nb_last = min(8, (__ldg(&J->width) - (tiles_x - 1) * kTileW) >> 4);
    r_job = __ldg(&J->param);
    c_t = t;
    return true;
  };
  auto step = [&]() -> bool {
    ++c_t;
    if (++tx == tiles_x) {
      tx = 0;
      src_band += (long long)kTileH * src_pitch;
      dst_band += (long long)kTileH * dst_pitch;
    }
    return c_t >= t_stop || c_t < c_end || enter(c_t);
  };
  bool ok = true;
  bool have = c_first + tau < c_stop;  // the cursor is on a tile of this warp
  if (have && !enter(c_first + tau)) ok = have = false;
  // The cursor's tile: its rows i16 of blocks p and p + 4 into staging slot
  // st (zeros for blocks past the image edge, read from nowhere); lane 0's
  // output row, the pitch, tile index, r and block count into the warp's ring
  // entry e; then the cursor moves two tiles on.  A warp without a tile
  // stages zeros, t = -1.
  auto take = [&](int e, int st) {
    unsigned char* d = tsm + kTcStage + st * 4096 + tid * 16;
    const uint8_t* dummy = reinterpret_cast<const uint8_t*>(jobs);
    if (have) {
      const int nb = tx == tiles_x - 1 ? nb_last : 8;
      const uint8_t* src = src_band + tx * kTileW;
      const unsigned long long dst = reinterpret_cast<unsigned long long>(dst_band + tx * kTileW);
      const int na = p < nb ? 16 : 0, nb4 = p + 4 < nb ? 16 : 0;
      cp_async16_zfill(d, na ? src : dummy, na);
      cp_async16_zfill(d + 2048, nb4 ? src + 64 : dummy, nb4);
      if (lane == 0) {
        ring[2 * e] = make_uint4((unsigned)dst, (unsigned)(dst >> 32), (unsigned)(c_t + t_shift),
                                 ((unsigned)r_job << 8) | (unsigned)nb);
        ring[2 * e + 1] = make_uint4((unsigned)dst_pitch, 0u, 0u, 0u);
      }
      ok = step() && ok;
      ok = step() && ok;
      have = ok && c_t < t_stop;
    } else {
      cp_async16_zfill(d, dummy, 0);
      cp_async16_zfill(d + 2048, dummy, 0);
      if (lane == 0) {
        ring[2 * e] = make_uint4(0u, 0u, 0xFFFFFFFFu, 0u);
        ring[2 * e + 1] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    cp_async_commit();
  };
  // staged pixels of slot st -> row tid of the pass-1 operand (block p in K
  // 0-15, block p + 4 in K 16-31)
  auto to_a1 = [&](int st) {
    const uint4 xa = *reinterpret_cast<const uint4*>(tsm + kTcStage + st * 4096 + tid * 16);
    const uint4 xb = *reinterpret_cast<const uint4*>(tsm + kTcStage + st * 4096 + 2048 + tid * 16);
    unsigned char* a = tsm + kTcA1 + (tid >> 3) * 512 + (tid & 7) * 16;
    store_row_f16(a, xa);
    store_row_f16(a + 256, xb);
  };
  // P (this thread's TMEM lane, columns 2 v + h) -> column m = i16 of the
  // pass-2 operand, rows (tau, p, v): v = 0..7 at a, v = 8..15 at a + 512,
  // block p + 4 at K + 16, i.e. + 256
  auto to_a2 = [&]() {
    float pv[32];
    tc::ld32(tlane, pv);
    tc::ld_wait();
    pv[0] -= 18432.0f;  // 16 * 1024 of the f16 pixels + 16 * 128: pixels centred at 128
    pv[1] -= 18432.0f;
    unsigned char* a = tsm + kTcA2 + (8 * tau + 2 * p) * 512 + (i16 >> 3) * 128 + (i16 & 7) * 16;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int g = 0; g < 2; ++g)
        *reinterpret_cast<uint4*>(a + 512 * g + 256 * h) =
            make_uint4(f16x2(pv[16 * g + 0 + h], pv[16 * g + 2 + h]), f16x2(pv[16 * g + 4 + h], pv[16 * g + 6 + h]),
                       f16x2(pv[16 * g + 8 + h], pv[16 * g + 10 + h]), f16x2(pv[16 * g + 12 + h], pv[16 * g + 14 + h]));
  };
  auto issue_mma1 = [&]() {
    tc::mma_f16(tbase + 0, dA1, dB1, idK, false);
    tc::mma_f16(tbase + 0, dA1 + kK16, dB1 + kK16, idK, true);
    tc::commit(bar1);
  };
  auto issue_mma2 = [&]() {
    tc::mma_f16(tbase + 32, dA2, dB2, idMN, false);
    tc::mma_f16(tbase + 32, dA2 + kK16, dB2 + kK16, idMN, true);
    tc::commit(bar2);
  };

  // ---- prologue: MMA2(0) and MMA1(1) in flight, the rows of pair 2 staged
  bool bad = false;
  take(0, 0);
  if (npairs > 1) {
    take(1, 1);
    cp_async_wait<1>();
  } else {
    cp_async_wait<0>();
  }
  to_a1(0);
  tc::fence_proxy_async();
  __syncthreads();
  if (tid == 0 && !stall) issue_mma1();  // stall: the failure-path test hook, no product ever arrives
  bad = !tc::mbar_wait(bar1, 0, kTcWaitCycles);
  tc::fence_after_sync();
  to_a2();
  if (npairs > 1) {
    cp_async_wait<0>();
    to_a1(1);
  }
  if (npairs > 2) take(2, 0);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  bad = __syncthreads_or(bad) != 0;
  if (tid == 0 && !bad) {
    tc::fence_after_sync();
    issue_mma2();
    if (npairs > 1) issue_mma1();
  }

  // the first warp of each tile finishes the tile's partial after the next barrier
  float own = 0.f;
  int own_t = -1;
  int wr = -1;  // r whose weights this warp holds
  float4* const wsm = reinterpret_cast<float4*>(tsm + kTcW) + warp * 144;
  for (int k = 0; k < npairs && !bad; ++k) {
    // ---- MMA2(k) and MMA1(k+1) complete: next operands, this pair's Y
    bool fail = !tc::mbar_wait(bar2, k & 1, kTcWaitCycles);
    tc::fence_after_sync();
    if (k + 1 < npairs) {
      fail = !tc::mbar_wait(bar1, (k + 1) & 1, kTcWaitCycles) || fail;
      tc::fence_after_sync();
      to_a2();
    }
    if (k + 2 < npairs) {
      cp_async_wait<0>();
      to_a1(k & 1);  // pair k + 2 sits in slot (k + 2) & 1
    }
    if (k + 3 < npairs) take((k + 3) & 3, (k + 1) & 1);
    float yv[32];  // column 2 u + h: 256 Y_c[u][v] of block p + 4 h
    tc::ld32(tlane + 32, yv);
    tc::ld_wait();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    bad = __syncthreads_or(fail) != 0;
    if (bad) break;
    if (tid == 0) {
      tc::fence_after_sync();
      if (k + 1 < npairs) issue_mma2();
      if (k + 2 < npairs) issue_mma1();
    }
    if ((warp & 1) == 0 && lane == 0 && own_t >= 0)
      tile_sse[own_t] = (own + part[2 * ((k - 1) & 1) + tau]) * (1.0f / (256.0f * 2304.0f));

    // ---- pair k on the CUDA cores: column v = i16 of blocks p, p + 4
    const uint4 md = ring[2 * (k & 3)];  // written by lane 0 three pairs ago (barriers since)
    const int cur_pitch = (int)ring[2 * (k & 3) + 1].x;
    const int cur_r = (int)(md.w >> 8), cur_nb = (int)(md.w & 255u);
    float2 y[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) y[u] = make_float2(yv[2 * u], yv[2 * u + 1]);
    if (i16 == 0) y[0] = badd(y[0], make_float2(8388608.0f, 8388608.0f));  // 256 Y_c -> 256 Y at (0, 0)
    float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    if (cur_r != wr) {  // warp-uniform (one tile per warp): refresh the warp's weight copy
      __syncwarp();
      const float4* const src = reinterpret_cast<const float4*>(wtab) + (long long)cur_r * 128;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int g = lane * 4 + q;
        wsm[9 * (g >> 3) + (g & 7)] = __ldg(src + g);  // (kw, dw) of rows 2h, 2h + 1 of column g >> 3
      }
      __syncwarp();
      wr = cur_r;
    }
    {
      const float4* const wcol = wsm + 9 * i16;
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const float4 w = wcol[h];  // (kw, dw) of rows 2h, 2h + 1 of column v
        acc = __ffma2_rn(f2mul(y[2 * h], w.y), y[2 * h], acc);
        acc1 = __ffma2_rn(f2mul(y[2 * h + 1], w.w), y[2 * h + 1], acc1);
        y[2 * h] = f2mul(y[2 * h], w.x);
        y[2 * h + 1] = f2mul(y[2 * h + 1], w.z);
      }
    }
    float2* const trb = reinterpret_cast<float2*>(tsm + kTcTr + warp * 4608) + (lane >> 4) * 288;
    {
      float2 uo[16];
      inv16(y, uo);
#pragma unroll
      for (int m = 0; m < 16; ++m) trb[18 * m + i16] = uo[m];
    }
    __syncwarp();
    {
      float2 v[16], z[16];
      const float4* const trr = reinterpret_cast<const float4*>(trb + 18 * i16);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 f = trr[q];
        v[2 * q] = make_float2(f.x, f.y);
        v[2 * q + 1] = make_float2(f.z, f.w);
      }
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
      // lane 0 holds row 0 of block pair 2 (warp & 1); this lane row i16 of pair p
      uint8_t* const dst = reinterpret_cast<uint8_t*>((unsigned long long)md.x | ((unsigned long long)md.y << 32)) +
                           (long long)i16 * cur_pitch + 16 * (lane >> 4);
      const bool va = p < cur_nb, vb = p + 4 < cur_nb;
      if (va) __stcs(reinterpret_cast<uint4*>(dst), make_uint4(oa[0], oa[1], oa[2], oa[3]));
      if (vb) __stcs(reinterpret_cast<uint4*>(dst + 64), make_uint4(ob[0], ob[1], ob[2], ob[3]));
      acc = __fadd2_rn(acc, acc1);
      const float tot = warp_sum((va ? acc.x : 0.f) + (vb ? acc.y : 0.f));
      if (warp & 1) {
        if (lane == 0) part[2 * (k & 1) + tau] = tot;
      } else {
        own = tot;
        own_t = (int)md.z;
      }
    }
  }

  // ---- the last pair's partials, then release TMEM
  cp_async_wait<0>();
  tc::fence_before_sync();
  bad = __syncthreads_or(bad) != 0;
  if (!bad && (warp & 1) == 0 && lane == 0 && own_t >= 0)
    tile_sse[own_t] = (own + part[2 * ((npairs - 1) & 1) + tau]) * (1.0f / (256.0f * 2304.0f));
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, kTcCols);
  }
  if (tid == 0 && bad) set_status(status, kDevTimeout);
  if (!ok && lane == 0) set_status(status, kDevBadJob);
  pdl_chain_exit();
}

cudaError_t launch_zonal_tc(const ImageJob* d_jobs, int njobs, long long ntiles, const float2* d_wtab,
                            float* d_tile_sse, int* d_status, int grid, cudaStream_t stream, bool dependent,
                            bool early, bool stall) {
  return launch_chained(zonal_tc_kernel, grid, 128, kTcSmemBytes, stream, dependent, d_jobs, njobs, ntiles, d_wtab,
                        d_tile_sse, d_status, early ? 1 : 0, stall ? 1 : 0);
}

// CTAs of the kernel that fit on one SM.  The occupancy calculator answers 1
// for a kernel that allocates tensor memory, while the SM co-schedules as
// many CTAs as registers, shared memory, threads and TMEM (64 of the 512
// columns per CTA) allow (4 on GB300, measured with a per-SM residency
// counter), so the count is derived from the kernel's attributes here.
int zonal_tc_max_ctas_per_sm() {
  cudaFuncAttributes fa;
  int dev = 0, regs = 0, smem = 0, reserved = 0, threads = 0;
  if (cudaFuncGetAttributes(&fa, zonal_tc_kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
    return 1;
  const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
  const int by_regs = regs / (4 * std::max(1, warp_regs));
  const int by_smem = smem / (kTcSmemBytes + (int)fa.sharedSizeBytes + reserved);
  const int by_threads = threads / 128;
  return std::max(1, std::min(std::min(by_regs, by_smem), std::min(by_threads, (int)(512 / kTcCols))));
}

}  // namespace atdct16
