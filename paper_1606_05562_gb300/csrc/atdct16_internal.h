// Internal declarations shared by the kernels and the C-ABI layer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace atdct16 {

// A tile is 16 image rows x 128 columns (eight 16x16 blocks).  One warp
// processes one tile at a time; the last tile of a row may hold fewer blocks.
constexpr int kTileW = 128;
constexpr int kTileH = 16;
constexpr int kZonalWarps = 4;  // warps per CTA of the fused zonal and quantisation kernels

// One image of a batch, as the kernels see it (64 bytes).
struct ImageJob {
  const uint8_t* src;
  uint8_t* dst;
  long long src_pitch;   // bytes
  long long dst_pitch;   // bytes
  long long tile_begin;  // first global tile index of this image
  long long level_base;  // quantisation path: first int16 level of this image
  int width;
  int height;
  int tiles_x;           // tiles per tile row = ceil(width / 128)
  int param;             // zonal r (0..256) or quantisation point QP (0..63)
};
static_assert(sizeof(ImageJob) == 64, "ImageJob layout");

// Zonal weights, one entry per (r, column c, row-frequency u):
// (kw, dw) = (keep, 1 - keep) * W_u * W_c / 256, W = 48 S^2 = 48 / diag(T T^T).
constexpr int kZonalTableEntries = 257 * 256;
// Quantiser constants per (QP, c, u): (k, s, g, Qstep) with s = s_u s_c,
// k = fp32(s / Qstep), g = fp32(s * Qstep).
constexpr int kMaxQP = 63;
constexpr int kQuantTableEntries = (kMaxQP + 1) * 256;

// Device status codes written by kernels' own checks (sticky, first wins).
constexpr int kDevOk = 0;
constexpr int kDevBadJob = 1;
constexpr int kDevTimeout = 2;  // a bounded wait on an asynchronous copy expired

// Kernel launchers (atdct16_kernels.cu).  All asynchronous on `stream`.
// The zonal launchers take a class-ordered table (see zonal_order below):
// the partial of a job's tile k goes to d_tile_sse[level_base + k].
// Launch shapes of the fused zonal kernel (chosen by the batch autotuner).
constexpr int kZonalF32 = 0;   // integer row pass, FP32 column pass and inverse
constexpr int kZonalSwar = 1;  // whole forward transform on the integer pipe (int16 SWAR)
constexpr int kZonalMma = 2;   // forward transform as f16 tensor-core products (exact), mma.sync
constexpr int kZonalTc = 3;    // forward transform as tcgen05 products with TMEM accumulators (exact)
struct ZonalConfig {
  int variant;   // kZonalF32, kZonalSwar, kZonalMma or kZonalTc
  int warps;     // warps per CTA: 2, 4 or 8 (SWAR: 4)
  int prefetch;  // 1: load the next tile while computing the current one
  int test_stall = 0;  // failure-path test hook: the tcgen05 variant issues no MMA, so its bounded waits expire
};
bool zonal_config_supported(const ZonalConfig& c);
ZonalConfig default_zonal_config();
int zonal_config_max_ctas_per_sm(const ZonalConfig& c);
// dependent: a programmatic dependent launch after the previous zonal kernel
// of the same call; early: let the next kernel be scheduled from the start.
cudaError_t launch_zonal_config(const ZonalConfig& cfg, const ImageJob* d_jobs, int njobs, long long ntiles,
                                const float2* d_wtab, float* d_tile_sse, int* d_status, int grid,
                                cudaStream_t stream, bool dependent = false, bool early = false);
// The tcgen05 variant (atdct16_zonal_tc.cu): one warpgroup per CTA.
cudaError_t launch_zonal_tc(const ImageJob* d_jobs, int njobs, long long ntiles, const float2* d_wtab,
                            float* d_tile_sse, int* d_status, int grid, cudaStream_t stream, bool dependent,
                            bool early, bool stall = false);
int zonal_tc_max_ctas_per_sm();
// d_levels (optional, 16-byte aligned): int16 levels per block, row-major
// in (u, v) or, with zigzag, in zig-zag order.
cudaError_t launch_quant(const ImageJob* d_jobs, int njobs, long long ntiles, const float4* d_qtab,
                         int16_t* d_levels, bool zigzag, float* d_tile_sse, int* d_status, int grid,
                         cudaStream_t stream);
cudaError_t launch_psnr_finalize(const ImageJob* d_jobs, int njobs, long long ntiles,
                                 const float* d_tile_sse, double peak, double* d_psnr,
                                 double* d_sse, cudaStream_t stream);
// Exact-DCT baseline of the fused zonal path (same tiles and table as zonal).
cudaError_t launch_zonal_dct(const ImageJob* d_jobs, int njobs, long long ntiles, const float2* d_wtab,
                             float* d_tile_sse, int* d_status, int num_sms, cudaStream_t stream);
// SSIM tiles: 20 x 128 window positions of an image's (h - 10) x (w - 10) map.
constexpr int kSsimTileRows = 20, kSsimTileCols = 128;
cudaError_t launch_ssim(const ImageJob* d_jobs, int njobs, long long ntiles, float* d_tile_sum, double* d_out,
                        int* d_status, int num_sms, cudaStream_t stream);
// Coefficient pipeline (atdct16_coef.cu): 2-D forward / exact inverse over
// 16x16 blocks (coefficients row-major in (u, v) or in zig-zag order) and
// 1-D forward / exact inverse over 16-sample vectors.
cudaError_t launch_forward(int dtype, const void* d_src, long long pitch, int w, int h, int32_t* d_coef,
                           bool zigzag, int num_sms, cudaStream_t stream);
cudaError_t launch_inverse(int dtype, const int32_t* d_coef, int w, int h, void* d_dst, long long pitch,
                           bool zigzag, int* d_status, unsigned extra_tx, int num_sms, cudaStream_t stream);
cudaError_t launch_forward_1d(int dtype, const void* d_src, long long count, int32_t* d_coef, int num_sms,
                              cudaStream_t stream);
cudaError_t launch_inverse_1d(int dtype, const int32_t* d_coef, long long count, void* d_dst, int num_sms,
                              cudaStream_t stream);
cudaError_t launch_psnr_pair(int dtype, const void* d_a, long long pitch_a, const void* d_b,
                             long long pitch_b, int w, int h, double* d_out, cudaStream_t stream);
int zonal_ctas_per_sm();

// Classes of zonal jobs (atdct16_zonal_box.cu).  A job whose kept zig-zag
// prefix lies in the K x K low-frequency corner (r <= K (K + 1) / 2, r >= 1)
// runs the box kernel of the smallest such K in kZonalBoxK; r = 0 and
// r > 36 run the general kernel.
constexpr int kZonalBoxClasses = 4;
constexpr int kZonalBoxK[kZonalBoxClasses] = {1, 3, 6, 8};
constexpr int kZonalGeneral = kZonalBoxClasses;
constexpr int kZonalClasses = kZonalBoxClasses + 1;
struct ZonalSplit {
  int first[kZonalClasses + 1];     // class c: jobs [first[c], first[c + 1]) of the class-ordered table
  long long ntiles[kZonalClasses];  // tiles of class c
};
int zonal_class_of(int r);
// Class-ordered copy of a zonal job table of n jobs: grouped by class (table
// order kept inside a class), each class's tiles numbered from 0 in
// tile_begin, and level_base = the job's tile_begin in `jobs` (where the
// kernels write its per-tile partials, which the PSNR finalize reads).
void zonal_order(const ImageJob* jobs, int n, ImageJob* ordered, ZonalSplit* split);
// Launch shape of the box kernels (the batch autotuner's knobs).
struct BoxConfig {
  int warps;        // warps per CTA, i.e. tiles per CTA in flight: 2, 4 or 8
  int depth;        // staging depth, tiles whose input rows are in flight per warp: 1, 2 or 3 (extent 8)
  int vec;          // bytes per input copy: 16 (one block row) or 8
  int ctas_per_sm;  // 0: as many as fit
};
bool box_config_supported(const BoxConfig& bc);
BoxConfig default_box_config();
int box_config_max_ctas_per_sm(const BoxConfig& bc);
// One launch per non-empty class on `stream`; `general` and `general_grid`
// shape the general kernel's launch, `box` the box kernels'.
cudaError_t launch_zonal_ordered(const ImageJob* d_ordered, const ZonalSplit& split, const ZonalConfig& general,
                                 int general_grid, const BoxConfig& box, const float2* d_wtab, float* d_tile_sse,
                                 int* d_status, int num_sms, cudaStream_t stream);

}  // namespace atdct16

// Plan internals shared with the batch layer (atdct16_api.cu).
struct atdct16_plan_st;
namespace atdct16 {
const float2* plan_zonal_table(const atdct16_plan_st* plan);
int plan_num_sms(const atdct16_plan_st* plan);
int plan_device(const atdct16_plan_st* plan);
bool plan_test_stall_mma(const atdct16_plan_st* plan);
bool plan_tune_lookup(atdct16_plan_st* plan, unsigned long long key, ZonalConfig* cfg, int* ctas, BoxConfig* box,
                      float* ms);
void plan_tune_store(atdct16_plan_st* plan, unsigned long long key, const ZonalConfig& cfg, int ctas,
                     const BoxConfig& box, float ms);
int quant_ctas_per_sm();

}  // namespace atdct16
