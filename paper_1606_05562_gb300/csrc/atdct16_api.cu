// C-ABI layer: plans, argument validation, host-side constant tables, launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/atdct16.h"
#include "atdct16_butterfly.cuh"
#include "atdct16_internal.h"
#include "atdct16_zigzag.cuh"

using namespace atdct16;

struct atdct16_plan_st {
  int device = 0;
  atdct16_dtype dtype = ATDCT16_U8;
  bool zigzag = false;                  // ATDCT16_PLAN_ZIGZAG: block coefficients / levels in zig-zag order
  bool stall_copies = false;            // ATDCT16_PLAN_TEST_STALL_COPIES (failure-path test hook)
  bool stall_mma = false;               // ATDCT16_PLAN_TEST_STALL_MMA (failure-path test hook)
  int max_images = 0;
  long long max_tiles = 0;
  int num_sms = 0;
  int zonal_grid = 0;
  int quant_grid = 0;
  ImageJob* d_jobs = nullptr;           // descriptors of the current call (one of d_jobs_buf[0..1])
  ImageJob* h_jobs = nullptr;           // pinned staging of the current call (one of h_jobs_buf[0..1])
  // Two descriptor buffers, used by alternate calls: the upload of a call's
  // descriptors runs on copy_stream while the previous call still computes.
  ImageJob* d_jobs_buf[2] = {nullptr, nullptr};
  ImageJob* h_jobs_buf[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t uploaded[2] = {nullptr, nullptr};  // upload of buffer b complete
  cudaEvent_t consumed[2] = {nullptr, nullptr};  // kernels reading buffer b complete
  bool uploaded_pending[2] = {false, false};
  bool consumed_pending[2] = {false, false};
  int buf = 1;                                   // buffer of the current call
  float2* d_wtab = nullptr;             // zonal weights [r][c][u]
  float4* d_qtab = nullptr;             // quantiser constants [QP][c][u]
  float* d_tile_sse = nullptr;          // per-tile SSE partials
  int* d_status = nullptr;
  cudaStream_t last_stream = nullptr;
  // autotuner results for this plan: batch-shape key -> (config, CTAs per SM, ms)
  struct Tuned {
    ZonalConfig cfg;
    int ctas;
    BoxConfig box;
    float ms;
  };
  std::map<unsigned long long, Tuned> tuned;
  // kernel timing hook
  bool profiling = false;
  int prof_every = 1;        // time one launch in prof_every
  long long prof_calls = 0;  // launches seen since profiling was enabled
  std::vector<cudaEvent_t> prof_events;  // pairs (start, stop)
  int prof_used = 0;                     // pairs recorded since the last query
};

namespace {

// Zig-zag rank of every (u, v) (Sec. 4): the inverse of the scan.
void zigzag_rank16(int rank[16][16]) {
  for (int k = 0; k < 256; ++k) {
    const int w = zigzag_word(k);
    rank[w >> 4][w & 15] = k;
  }
}

constexpr int kProfPairs = 4096;

// Start / stop events around one kernel launch when profiling is on.
int prof_begin(atdct16_plan_t plan, cudaStream_t stream) {
  if (!plan->profiling || plan->prof_used >= kProfPairs) return -1;
  if (plan->prof_calls++ % plan->prof_every != 0) return -1;
  const int k = plan->prof_used++;
  if (cudaEventRecord(plan->prof_events[2 * k], stream) != cudaSuccess) return -1;
  return k;
}
void prof_end(atdct16_plan_t plan, int k, cudaStream_t stream) {
  if (k >= 0) cudaEventRecord(plan->prof_events[2 * k + 1], stream);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

atdct16_status from_cuda(cudaError_t e) { return e == cudaSuccess ? ATDCT16_OK : ATDCT16_ECUDA; }

atdct16_status check_image(const atdct16_image& im, int elem, bool need_dst) {
  if (!im.src || (need_dst && !im.dst)) return ATDCT16_EINVAL;
  if (im.width <= 0 || im.height <= 0 || (im.width & 15) || (im.height & 15)) return ATDCT16_EINVAL;
  if (im.src_pitch < (int64_t)im.width * elem || (im.src_pitch & 15)) return ATDCT16_EINVAL;
  if (need_dst && (im.dst_pitch < (int64_t)im.width * elem || (im.dst_pitch & 15))) return ATDCT16_EINVAL;
  if (!aligned16(im.src) || (need_dst && !aligned16(im.dst))) return ATDCT16_EINVAL;
  if (im.reserved != 0) return ATDCT16_EINVAL;
  if (im.src_pitch >= ((int64_t)1 << 31) || im.dst_pitch >= ((int64_t)1 << 31)) return ATDCT16_EINVAL;
  return ATDCT16_OK;
}

// Fill a pinned descriptor staging buffer and upload it.  Calls alternate
// between two buffers; the upload runs on the plan's copy stream (so it
// overlaps the previous call's kernels) and `stream` waits for it.  While
// `stream` is being captured into a graph the upload goes on `stream` itself.
atdct16_status stage_jobs(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n, int elem,
                          cudaStream_t stream, long long* ntiles_out, bool with_level_base, bool ssim_tiles = false,
                          ZonalSplit* zonal_split = nullptr) {
  const int b = plan->buf ^ 1;
  if (plan->uploaded_pending[b]) {
    if (cudaEventSynchronize(plan->uploaded[b]) != cudaSuccess) return ATDCT16_ECUDA;
    plan->uploaded_pending[b] = false;
  }
  ImageJob* const hj = plan->h_jobs_buf[b];
  long long tiles = 0, blocks = 0;
  for (int i = 0; i < n; ++i) {
    const atdct16_image& im = h_images[i];
    ImageJob& J = hj[i];
    J.src = static_cast<const uint8_t*>(im.src);
    J.dst = static_cast<uint8_t*>(im.dst);
    J.src_pitch = im.src_pitch;
    J.dst_pitch = im.dst_pitch;
    J.width = im.width;
    J.height = im.height;
    J.param = im.r_or_qp;
    J.tile_begin = tiles;
    if (ssim_tiles) {  // tiles of the (h - 10) x (w - 10) map of window positions
      J.tiles_x = (im.width - 10 + kSsimTileCols - 1) / kSsimTileCols;
      tiles += (long long)J.tiles_x * ((im.height - 10 + kSsimTileRows - 1) / kSsimTileRows);
    } else {
      J.tiles_x = (im.width + kTileW - 1) / kTileW;
      tiles += (long long)J.tiles_x * (im.height / kTileH);
    }
    J.level_base = with_level_base ? blocks * 256 : 0;
    blocks += (long long)(im.width / 16) * (im.height / 16);
  }
  if (tiles > plan->max_tiles) return ATDCT16_ENOMEM;
  // zonal calls: the class-ordered copy for the kernels follows the table
  if (zonal_split) zonal_order(hj, n, hj + n, zonal_split);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return ATDCT16_ECUDA;
  const size_t bytes = sizeof(ImageJob) * n * (zonal_split ? 2 : 1);
  cudaError_t e = cudaSuccess;
  if (cap == cudaStreamCaptureStatusNone) {
    if (plan->consumed_pending[b]) e = cudaStreamWaitEvent(plan->copy_stream, plan->consumed[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan->d_jobs_buf[b], hj, bytes, cudaMemcpyHostToDevice, plan->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(plan->uploaded[b], plan->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, plan->uploaded[b], 0);
    if (e != cudaSuccess) return ATDCT16_ECUDA;
    plan->uploaded_pending[b] = true;
  } else {
    // inside a capture: everything on the capturing stream, after any work
    // still reading this buffer has drained
    if (plan->consumed_pending[b] && cudaEventSynchronize(plan->consumed[b]) != cudaSuccess) return ATDCT16_ECUDA;
    e = cudaMemcpyAsync(plan->d_jobs_buf[b], hj, bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return ATDCT16_ECUDA;
  }
  plan->consumed_pending[b] = false;
  plan->buf = b;
  plan->d_jobs = plan->d_jobs_buf[b];
  plan->h_jobs = hj;
  plan->last_stream = stream;
  *ntiles_out = tiles;
  (void)elem;
  return ATDCT16_OK;
}

// After the kernels that read the current descriptor buffer are enqueued.
void jobs_consumed(atdct16_plan_t plan, cudaStream_t stream) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
  if (cudaEventRecord(plan->consumed[plan->buf], stream) == cudaSuccess) plan->consumed_pending[plan->buf] = true;
}

}  // namespace

namespace atdct16 {
const float2* plan_zonal_table(const atdct16_plan_st* plan) { return plan->d_wtab; }
int plan_num_sms(const atdct16_plan_st* plan) { return plan->num_sms; }
int plan_device(const atdct16_plan_st* plan) { return plan->device; }
bool plan_test_stall_mma(const atdct16_plan_st* plan) { return plan->stall_mma; }
bool plan_tune_lookup(atdct16_plan_st* plan, unsigned long long key, ZonalConfig* cfg, int* ctas, BoxConfig* box,
                      float* ms) {
  auto it = plan->tuned.find(key);
  if (it == plan->tuned.end()) return false;
  *cfg = it->second.cfg;
  *ctas = it->second.ctas;
  *box = it->second.box;
  *ms = it->second.ms;
  return true;
}
void plan_tune_store(atdct16_plan_st* plan, unsigned long long key, const ZonalConfig& cfg, int ctas,
                     const BoxConfig& box, float ms) {
  plan->tuned[key] = atdct16_plan_st::Tuned{cfg, ctas, box, ms};
}
}  // namespace atdct16

extern "C" {

const char* atdct16_version(void) { return "atdct16 1.0 sm_103a"; }

const char* atdct16_status_string(atdct16_status s) {
  switch (s) {
    case ATDCT16_OK: return "ok";
    case ATDCT16_EINVAL: return "invalid argument";
    case ATDCT16_ENOMEM: return "out of workspace or device memory";
    case ATDCT16_ECUDA: return "CUDA runtime error";
    case ATDCT16_ETIMEOUT: return "device-side wait timed out";
    case ATDCT16_EUNSUPPORTED: return "unsupported request";
    case ATDCT16_EDEVICE: return "kernel rejected a descriptor";
  }
  return "unknown status";
}

atdct16_status atdct16_host_butterfly(const int32_t* in, int32_t* out, int32_t inverse) {
  if (!in || !out) return ATDCT16_EINVAL;
  int x[16], y[16];
  for (int i = 0; i < 16; ++i) x[i] = in[i];
  if (inverse) inv16(x, y); else fwd16(x, y);
  for (int i = 0; i < 16; ++i) out[i] = y[i];
  return ATDCT16_OK;
}

atdct16_status atdct16_plan_destroy(atdct16_plan_t plan) {
  if (!plan) return ATDCT16_EINVAL;
  cudaSetDevice(plan->device);
  if (plan->last_stream) cudaStreamSynchronize(plan->last_stream);
  if (plan->copy_stream) cudaStreamSynchronize(plan->copy_stream);
  cudaFree(plan->d_jobs_buf[0]);
  cudaFree(plan->d_wtab);
  cudaFree(plan->d_qtab);
  cudaFree(plan->d_tile_sse);
  cudaFree(plan->d_status);
  cudaFreeHost(plan->h_jobs_buf[0]);
  for (int b = 0; b < 2; ++b) {
    if (plan->uploaded[b]) cudaEventDestroy(plan->uploaded[b]);
    if (plan->consumed[b]) cudaEventDestroy(plan->consumed[b]);
  }
  if (plan->copy_stream) cudaStreamDestroy(plan->copy_stream);
  for (cudaEvent_t ev : plan->prof_events) cudaEventDestroy(ev);
  delete plan;
  return ATDCT16_OK;
}

atdct16_status atdct16_plan_create(atdct16_plan_t* out, atdct16_dtype dtype, int32_t max_images,
                                   size_t workspace_budget_bytes, uint32_t flags) {
  if (!out || max_images < 1 || (flags & ~(ATDCT16_PLAN_ZIGZAG | ATDCT16_PLAN_TEST_STALL_COPIES | ATDCT16_PLAN_TEST_STALL_MMA)) != 0 || (dtype != ATDCT16_U8 && dtype != ATDCT16_I16))
    return ATDCT16_EINVAL;
  *out = nullptr;
  atdct16_plan_st* plan = new (std::nothrow) atdct16_plan_st();
  if (!plan) return ATDCT16_ENOMEM;
  plan->dtype = dtype;
  plan->zigzag = (flags & ATDCT16_PLAN_ZIGZAG) != 0;
  plan->stall_copies = (flags & ATDCT16_PLAN_TEST_STALL_COPIES) != 0;
  plan->stall_mma = (flags & ATDCT16_PLAN_TEST_STALL_MMA) != 0;
  plan->max_images = max_images;
  if (cudaGetDevice(&plan->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&plan->num_sms, cudaDevAttrMultiProcessorCount, plan->device) != cudaSuccess) {
    delete plan;
    return ATDCT16_ECUDA;
  }
  const size_t budget = workspace_budget_bytes ? workspace_budget_bytes : (size_t)256 << 20;
  const size_t fixed = 4 * sizeof(ImageJob) * max_images +
                       sizeof(float2) * kZonalTableEntries + sizeof(float4) * kQuantTableEntries + 256;
  if (budget <= fixed + 1024 * sizeof(float)) {
    delete plan;
    return ATDCT16_ENOMEM;
  }
  plan->max_tiles = (long long)((budget - fixed) / sizeof(float));

  // Host tables.  S^2 = 1 / nnz(row of T) (T T^T is diagonal with the row
  // non-zero counts, Sec. 2), so W = 48 S^2 = 48 / nnz.
  int nnz[16], rank[16][16];
  row_nonzeros(nnz);
  zigzag_rank16(rank);
  std::vector<float2> wtab(kZonalTableEntries);
  for (int r = 0; r <= 256; ++r)
    for (int c = 0; c < 16; ++c)
      for (int u = 0; u < 16; ++u) {
        const double wgt = (48.0 / nnz[u]) * (48.0 / nnz[c]) / 256.0;  // exact in FP32
        const bool keep = rank[u][c] < r;
        wtab[(r * 16 + c) * 16 + u] = make_float2(keep ? (float)wgt : 0.f, keep ? 0.f : (float)wgt);
      }
  std::vector<float4> qtab(kQuantTableEntries);
  for (int qp = 0; qp <= kMaxQP; ++qp) {
    const double qs = std::pow(2.0, qp / 6.0);
    for (int c = 0; c < 16; ++c)
      for (int u = 0; u < 16; ++u) {
        // s_u s_v as the product of the two FP64 diagonal entries of S
        const double s = (1.0 / std::sqrt((double)nnz[u])) * (1.0 / std::sqrt((double)nnz[c]));
        qtab[(qp * 16 + c) * 16 + u] = make_float4((float)(s / qs), (float)s, (float)(s * qs), (float)qs);
      }
  }

  cudaError_t e = cudaSuccess;
  // two descriptor buffers of 2 max_images each: a zonal call stores its
  // table followed by the class-ordered copy the kernels read
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_jobs_buf[0], 4 * sizeof(ImageJob) * max_images);
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_wtab, sizeof(float2) * kZonalTableEntries);
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_qtab, sizeof(float4) * kQuantTableEntries);
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_tile_sse, sizeof(float) * plan->max_tiles);
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaHostAlloc(&plan->h_jobs_buf[0], 4 * sizeof(ImageJob) * max_images, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&plan->uploaded[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->consumed[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) {
    plan->d_jobs_buf[1] = plan->d_jobs_buf[0] + 2 * max_images;
    plan->h_jobs_buf[1] = plan->h_jobs_buf[0] + 2 * max_images;
    plan->d_jobs = plan->d_jobs_buf[0];
    plan->h_jobs = plan->h_jobs_buf[0];
  }
  if (e == cudaSuccess) e = cudaMemcpy(plan->d_wtab, wtab.data(), sizeof(float2) * kZonalTableEntries, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(plan->d_qtab, qtab.data(), sizeof(float4) * kQuantTableEntries, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(plan->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    atdct16_plan_destroy(plan);
    return e == cudaErrorMemoryAllocation ? ATDCT16_ENOMEM : ATDCT16_ECUDA;
  }
  plan->zonal_grid = plan->num_sms * zonal_ctas_per_sm();
  plan->quant_grid = plan->num_sms * quant_ctas_per_sm();
  *out = plan;
  return ATDCT16_OK;
}

atdct16_status atdct16_forward(atdct16_plan_t plan, atdct16_dtype dtype, const void* d_src, int64_t pitch,
                               int32_t w, int32_t h, int32_t* d_coef, cudaStream_t stream) {
  if (!plan || !d_src || !d_coef || (dtype != ATDCT16_U8 && dtype != ATDCT16_I16)) return ATDCT16_EINVAL;
  const int elem = dtype == ATDCT16_U8 ? 1 : 2;
  if (w <= 0 || h <= 0 || (w & 15) || (h & 15) || pitch < (int64_t)w * elem || (pitch & 15)) return ATDCT16_EINVAL;
  if (!aligned16(d_src) || !aligned16(d_coef)) return ATDCT16_EINVAL;
  plan->last_stream = stream;
  return from_cuda(launch_forward(dtype, d_src, pitch, w, h, d_coef, plan->zigzag, plan->num_sms, stream));
}

atdct16_status atdct16_inverse(atdct16_plan_t plan, atdct16_dtype dtype, const int32_t* d_coef, int32_t w,
                               int32_t h, void* d_dst, int64_t pitch, cudaStream_t stream) {
  if (!plan || !d_dst || !d_coef || (dtype != ATDCT16_U8 && dtype != ATDCT16_I16)) return ATDCT16_EINVAL;
  const int elem = dtype == ATDCT16_U8 ? 1 : 2;
  if (w <= 0 || h <= 0 || (w & 15) || (h & 15) || pitch < (int64_t)w * elem || (pitch & 15)) return ATDCT16_EINVAL;
  if (!aligned16(d_dst) || !aligned16(d_coef)) return ATDCT16_EINVAL;
  plan->last_stream = stream;
  return from_cuda(
      launch_inverse(dtype, d_coef, w, h, d_dst, pitch, plan->zigzag, plan->d_status, plan->stall_copies ? 16u : 0u,
                     plan->num_sms, stream));
}

atdct16_status atdct16_forward_1d(atdct16_plan_t plan, atdct16_dtype dtype, const void* d_src, int64_t count,
                                  int32_t* d_coef, cudaStream_t stream) {
  if (!plan || count < 0 || (dtype != ATDCT16_U8 && dtype != ATDCT16_I16)) return ATDCT16_EINVAL;
  if (count == 0) return ATDCT16_OK;
  if (!d_src || !d_coef || !aligned16(d_src) || !aligned16(d_coef)) return ATDCT16_EINVAL;
  plan->last_stream = stream;
  return from_cuda(launch_forward_1d(dtype, d_src, count, d_coef, plan->num_sms, stream));
}

atdct16_status atdct16_inverse_1d(atdct16_plan_t plan, atdct16_dtype dtype, const int32_t* d_coef, int64_t count,
                                  void* d_dst, cudaStream_t stream) {
  if (!plan || count < 0 || (dtype != ATDCT16_U8 && dtype != ATDCT16_I16)) return ATDCT16_EINVAL;
  if (count == 0) return ATDCT16_OK;
  if (!d_coef || !d_dst || !aligned16(d_coef) || !aligned16(d_dst)) return ATDCT16_EINVAL;
  plan->last_stream = stream;
  return from_cuda(launch_inverse_1d(dtype, d_coef, count, d_dst, plan->num_sms, stream));
}

atdct16_status atdct16_compress_zonal(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n,
                                      double* d_psnr, double* d_sse, cudaStream_t stream) {
  if (!plan || !h_images || !d_psnr || n < 1 || n > plan->max_images) return ATDCT16_EINVAL;
  for (int i = 0; i < n; ++i) {
    const atdct16_status s = check_image(h_images[i], 1, true);
    if (s != ATDCT16_OK) return s;
    if (h_images[i].r_or_qp < 0 || h_images[i].r_or_qp > 256) return ATDCT16_EINVAL;
  }
  long long ntiles = 0;
  ZonalSplit split;
  atdct16_status s = stage_jobs(plan, h_images, n, 1, stream, &ntiles, false, false, &split);
  if (s != ATDCT16_OK) return s;
  const int pk = prof_begin(plan, stream);
  cudaError_t e = launch_zonal_ordered(plan->d_jobs + n, split, default_zonal_config(), plan->zonal_grid,
                                       default_box_config(), plan->d_wtab, plan->d_tile_sse, plan->d_status,
                                       plan->num_sms, stream);
  prof_end(plan, pk, stream);
  if (e == cudaSuccess)
    e = launch_psnr_finalize(plan->d_jobs, n, ntiles, plan->d_tile_sse, 255.0, d_psnr, d_sse, stream);
  if (e == cudaSuccess) jobs_consumed(plan, stream);
  return from_cuda(e);
}

atdct16_status atdct16_compress_quant(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n,
                                      int16_t* d_levels, double* d_psnr, double* d_sse, cudaStream_t stream) {
  if (!plan || !h_images || !d_psnr || n < 1 || n > plan->max_images) return ATDCT16_EINVAL;
  for (int i = 0; i < n; ++i) {
    const atdct16_status s = check_image(h_images[i], 2, true);
    if (s != ATDCT16_OK) return s;
    if (h_images[i].r_or_qp < 0 || h_images[i].r_or_qp > kMaxQP) return ATDCT16_EINVAL;
  }
  if (d_levels && !aligned16(d_levels)) return ATDCT16_EINVAL;
  long long ntiles = 0;
  atdct16_status s = stage_jobs(plan, h_images, n, 2, stream, &ntiles, d_levels != nullptr);
  if (s != ATDCT16_OK) return s;
  const int grid = (int)std::min<long long>(plan->quant_grid, (ntiles + kZonalWarps - 1) / kZonalWarps);
  const int pk = prof_begin(plan, stream);
  cudaError_t e = launch_quant(plan->d_jobs, n, ntiles, plan->d_qtab, d_levels, plan->zigzag, plan->d_tile_sse,
                               plan->d_status, grid, stream);
  prof_end(plan, pk, stream);
  if (e == cudaSuccess)
    e = launch_psnr_finalize(plan->d_jobs, n, ntiles, plan->d_tile_sse, 255.0, d_psnr, d_sse, stream);
  if (e == cudaSuccess) jobs_consumed(plan, stream);
  return from_cuda(e);
}

atdct16_status atdct16_compress_zonal_dct(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n,
                                          double* d_psnr, double* d_sse, cudaStream_t stream) {
  if (!plan || !h_images || !d_psnr || n < 1 || n > plan->max_images) return ATDCT16_EINVAL;
  for (int i = 0; i < n; ++i) {
    const atdct16_status s = check_image(h_images[i], 1, true);
    if (s != ATDCT16_OK) return s;
    if (h_images[i].r_or_qp < 0 || h_images[i].r_or_qp > 256) return ATDCT16_EINVAL;
  }
  long long ntiles = 0;
  atdct16_status s = stage_jobs(plan, h_images, n, 1, stream, &ntiles, false);
  if (s != ATDCT16_OK) return s;
  const int pk = prof_begin(plan, stream);
  cudaError_t e = launch_zonal_dct(plan->d_jobs, n, ntiles, plan->d_wtab, plan->d_tile_sse, plan->d_status,
                                   plan->num_sms, stream);
  prof_end(plan, pk, stream);
  if (e == cudaSuccess)
    e = launch_psnr_finalize(plan->d_jobs, n, ntiles, plan->d_tile_sse, 255.0, d_psnr, d_sse, stream);
  if (e == cudaSuccess) jobs_consumed(plan, stream);
  return from_cuda(e);
}

atdct16_status atdct16_ssim_batch(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n, double* d_mssim,
                                  cudaStream_t stream) {
  if (!plan || !h_images || !d_mssim || n < 1 || n > plan->max_images) return ATDCT16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_mssim) & 7) != 0) return ATDCT16_EINVAL;
  for (int i = 0; i < n; ++i) {
    const atdct16_status s = check_image(h_images[i], 1, true);
    if (s != ATDCT16_OK) return s;
  }
  long long ntiles = 0;
  atdct16_status s = stage_jobs(plan, h_images, n, 1, stream, &ntiles, false, true);
  if (s != ATDCT16_OK) return s;
  cudaError_t e = launch_ssim(plan->d_jobs, n, ntiles, plan->d_tile_sse, d_mssim, plan->d_status, plan->num_sms,
                              stream);
  if (e == cudaSuccess) jobs_consumed(plan, stream);
  return from_cuda(e);
}

atdct16_status atdct16_psnr(atdct16_dtype dtype, const void* d_a, int64_t pitch_a, const void* d_b,
                            int64_t pitch_b, int32_t w, int32_t h, double* d_out, cudaStream_t stream) {
  if (!d_a || !d_b || !d_out || (dtype != ATDCT16_U8 && dtype != ATDCT16_I16)) return ATDCT16_EINVAL;
  const int elem = dtype == ATDCT16_U8 ? 1 : 2;
  if (w <= 0 || h <= 0 || pitch_a < (int64_t)w * elem || pitch_b < (int64_t)w * elem) return ATDCT16_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_out) & 7) != 0) return ATDCT16_EINVAL;
  if (elem == 2 && ((pitch_a | pitch_b) & 1)) return ATDCT16_EINVAL;
  return from_cuda(launch_psnr_pair(dtype, d_a, pitch_a, d_b, pitch_b, w, h, d_out, stream));
}

atdct16_status atdct16_plan_set_profiling(atdct16_plan_t plan, int32_t every) {
  if (!plan || every < 0) return ATDCT16_EINVAL;
  if (every && plan->prof_events.empty()) {
    plan->prof_events.resize(2 * kProfPairs, nullptr);
    for (auto& ev : plan->prof_events)
      if (cudaEventCreate(&ev) != cudaSuccess) return ATDCT16_ECUDA;
  }
  plan->profiling = every != 0;
  plan->prof_every = every > 0 ? every : 1;
  plan->prof_calls = 0;
  plan->prof_used = 0;
  return ATDCT16_OK;
}

atdct16_status atdct16_plan_profile(atdct16_plan_t plan, int64_t* launches, double* kernel_ms) {
  if (!plan || !launches || !kernel_ms) return ATDCT16_EINVAL;
  double total = 0.0;
  for (int k = 0; k < plan->prof_used; ++k) {
    float ms = 0.f;
    if (cudaEventSynchronize(plan->prof_events[2 * k + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, plan->prof_events[2 * k], plan->prof_events[2 * k + 1]) != cudaSuccess)
      return ATDCT16_ECUDA;
    total += ms;
  }
  *launches = plan->prof_used;
  *kernel_ms = total;
  plan->prof_used = 0;
  return ATDCT16_OK;
}

atdct16_status atdct16_last_device_status(atdct16_plan_t plan) {
  if (!plan) return ATDCT16_EINVAL;
  if (plan->last_stream && cudaStreamSynchronize(plan->last_stream) != cudaSuccess) return ATDCT16_ECUDA;
  int v = 0;
  if (cudaMemcpy(&v, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ATDCT16_ECUDA;
  return v == kDevOk ? ATDCT16_OK : (v == kDevTimeout ? ATDCT16_ETIMEOUT : ATDCT16_EDEVICE);
}

}  // extern "C"
