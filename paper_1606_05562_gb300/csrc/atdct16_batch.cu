// Resident batches: descriptors uploaded once, launch shape autotuned on the
// batch itself, fused zonal kernel + PSNR finalize captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/atdct16.h"
#include "atdct16_internal.h"

using namespace atdct16;

struct atdct16_batch_st {
  atdct16_plan_t plan = nullptr;
  int device = 0;
  int n = 0;
  long long ntiles = 0;
  ImageJob* d_jobs = nullptr;  // the table (n jobs), then its class-ordered copy (n jobs)
  ZonalSplit split{};
  float* d_tile_sse = nullptr;
  int* d_status = nullptr;
  double* d_psnr = nullptr;
  double* d_sse = nullptr;
  ZonalConfig cfg{};
  int ctas = 1;
  int grid = 1;
  BoxConfig box{};
  float tuned_ms = 0.f;
  std::vector<atdct16_tune_point> cands;  // every launch shape the autotuner timed
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t last_stream = nullptr;
};

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

atdct16_status check_zonal_image(const atdct16_image& im) {
  if (!im.src || !im.dst || im.width <= 0 || im.height <= 0 || (im.width & 15) || (im.height & 15))
    return ATDCT16_EINVAL;
  if (im.src_pitch < im.width || im.dst_pitch < im.width || (im.src_pitch & 15) || (im.dst_pitch & 15))
    return ATDCT16_EINVAL;
  if (im.src_pitch >= ((int64_t)1 << 31) || im.dst_pitch >= ((int64_t)1 << 31)) return ATDCT16_EINVAL;
  if (!aligned16(im.src) || !aligned16(im.dst) || im.reserved != 0 || im.r_or_qp < 0 || im.r_or_qp > 256)
    return ATDCT16_EINVAL;
  return ATDCT16_OK;
}

// Does any destination byte range overlap any source byte range?
bool dst_overlaps_src(const atdct16_image* im, int n) {
  struct Range {
    uintptr_t lo, hi;
    int kind;  // 0 src, 1 dst
  };
  std::vector<Range> r;
  r.reserve(2 * n);
  for (int i = 0; i < n; ++i) {
    const uintptr_t s = reinterpret_cast<uintptr_t>(im[i].src), d = reinterpret_cast<uintptr_t>(im[i].dst);
    r.push_back({s, s + (uintptr_t)im[i].src_pitch * (im[i].height - 1) + im[i].width, 0});
    r.push_back({d, d + (uintptr_t)im[i].dst_pitch * (im[i].height - 1) + im[i].width, 1});
  }
  std::sort(r.begin(), r.end(), [](const Range& a, const Range& b) { return a.lo < b.lo; });
  // sweep: any open range of the other kind reaching past this start overlaps
  uintptr_t max_hi[2] = {0, 0};
  for (const Range& x : r) {
    if (max_hi[1 - x.kind] > x.lo) return true;
    max_hi[x.kind] = std::max(max_hi[x.kind], x.hi);
  }
  return false;
}

// FNV-1a over the batch shape: sizes, r and the device's SM count.
unsigned long long shape_key(const atdct16_image* im, int n, int sms) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xff;
      h *= 1099511628211ull;
    }
  };
  mix((unsigned long long)n);
  mix((unsigned long long)sms);
  for (int i = 0; i < n; ++i) {
    mix((unsigned long long)im[i].width << 32 | (unsigned)im[i].height);
    mix((unsigned long long)im[i].r_or_qp);
  }
  return h;
}

int grid_for(const ZonalConfig& cfg, int ctas, int sms, long long ntiles) {
  const long long need = (ntiles + cfg.warps - 1) / cfg.warps;
  return (int)std::max<long long>(1, std::min<long long>((long long)sms * ctas, need));
}

// Tuning-cache file (ATDCT16_TUNE_CACHE): one JSON object per line,
// {"key": "<hex>", "variant": v, "warps": w, "prefetch": p, "ctas": c, "tiles_per_cta": W,
//  "staging_depth": D, "vector_bytes": V, "box_ctas": B, "ms": t}
bool file_lookup(unsigned long long key, ZonalConfig* cfg, int* ctas, BoxConfig* box, float* ms) {
  const char* path = std::getenv("ATDCT16_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    unsigned long long k = 0;
    int v, w, p, c, bw, bd, bv, bc;
    float t;
    if (std::sscanf(line,
                    " {\"key\": \"%llx\", \"variant\": %d, \"warps\": %d, \"prefetch\": %d, \"ctas\": %d, "
                    "\"tiles_per_cta\": %d, \"staging_depth\": %d, \"vector_bytes\": %d, \"box_ctas\": %d, \"ms\": %f",
                    &k, &v, &w, &p, &c, &bw, &bd, &bv, &bc, &t) == 10 &&
        k == key) {
      const ZonalConfig z{v, w, p};
      const BoxConfig b{bw, bd, bv, bc};
      if (zonal_config_supported(z) && c >= 1 && box_config_supported(b)) {
        *cfg = z;
        *ctas = c;
        *box = b;
        *ms = t;
        found = true;  // the last matching line wins
      }
    }
  }
  std::fclose(f);
  return found;
}

void file_store(unsigned long long key, const ZonalConfig& cfg, int ctas, const BoxConfig& box, float ms) {
  const char* path = std::getenv("ATDCT16_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f,
               "{\"key\": \"%016llx\", \"variant\": %d, \"warps\": %d, \"prefetch\": %d, \"ctas\": %d, "
               "\"tiles_per_cta\": %d, \"staging_depth\": %d, \"vector_bytes\": %d, \"box_ctas\": %d, \"ms\": %.6f}\n",
               key, cfg.variant, cfg.warps, cfg.prefetch, ctas, box.warps, box.depth, box.vec, box.ctas_per_sm, ms);
  std::fclose(f);
}

cudaError_t launch_batch_once(atdct16_batch_st* b, const ZonalConfig& cfg, int grid, const BoxConfig& box,
                              cudaStream_t stream) {
  cudaError_t e = launch_zonal_ordered(b->d_jobs + b->n, b->split, cfg, grid, box, plan_zonal_table(b->plan),
                                       b->d_tile_sse, b->d_status, plan_num_sms(b->plan), stream);
  if (e == cudaSuccess)
    e = launch_psnr_finalize(b->d_jobs, b->n, b->ntiles, b->d_tile_sse, 255.0, b->d_psnr, b->d_sse, stream);
  return e;
}

// Median time of one launch of the batch in a given shape: a warm-up launch,
// then kTuneReps launches each between two events.
constexpr int kTuneReps = 5;
atdct16_status time_shape(atdct16_batch_st* b, const ZonalConfig& cfg, int grid, const BoxConfig& box,
                          cudaStream_t stream, cudaEvent_t e0, cudaEvent_t e1, float* ms_out) {
  if (launch_batch_once(b, cfg, grid, box, stream) != cudaSuccess) return ATDCT16_ECUDA;
  float t[kTuneReps];
  for (int rep = 0; rep < kTuneReps; ++rep) {
    if (cudaEventRecord(e0, stream) != cudaSuccess || launch_batch_once(b, cfg, grid, box, stream) != cudaSuccess ||
        cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t[rep], e0, e1) != cudaSuccess)
      return ATDCT16_ECUDA;
  }
  std::sort(t, t + kTuneReps);
  *ms_out = t[kTuneReps / 2];
  return ATDCT16_OK;
}

atdct16_tune_point tune_point(const ZonalConfig& cfg, int ctas, const BoxConfig& box, float ms, int phase = 0) {
  atdct16_tune_point t;
  t.phase = phase;
  t.variant = cfg.variant;
  t.general_ctas = ctas;
  t.tiles_per_cta = box.warps;
  t.staging_depth = box.depth;
  t.vector_bytes = box.vec;
  t.box_ctas = box.ctas_per_sm;
  t.ms = ms;
  return t;
}

// Autotuner.  Box kernels (jobs with r <= 36): tiles per CTA (warps) in
// {2, 4, 8} x staging depth {1, 2, 3} x input copy width {16, 8} bytes x
// CTAs per SM {as many as fit, half}; then, if the batch has jobs for the
// general kernel, its variant x CTAs per SM with the box shape found.  Each
// candidate is the median of five timed launches of the whole batch.
atdct16_status autotune(atdct16_batch_st* b, int sms, cudaStream_t stream) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return ATDCT16_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ATDCT16_ECUDA;
  }
  bool has_box = false;
  for (int c = 0; c < kZonalBoxClasses; ++c) has_box = has_box || b->split.ntiles[c] > 0;
  const bool has_general = b->split.ntiles[kZonalGeneral] > 0;
  ZonalConfig best_cfg = default_zonal_config();
  int best_ctas = zonal_config_max_ctas_per_sm(best_cfg);
  BoxConfig best_box = default_box_config();
  float best = 1e30f;
  atdct16_status st = ATDCT16_OK;
  b->cands.clear();
  if (has_box) {
    const int warps[3] = {2, 4, 8}, depths[3] = {1, 2, 3}, vecs[2] = {16, 8};
    for (int wi = 0; wi < 3 && st == ATDCT16_OK; ++wi)
      for (int di = 0; di < 3 && st == ATDCT16_OK; ++di)
        for (int vi = 0; vi < 2 && st == ATDCT16_OK; ++vi) {
          BoxConfig bc{warps[wi], depths[di], vecs[vi], 0};
          const int maxc = box_config_max_ctas_per_sm(bc);
          for (int half = 0; half < (maxc > 1 ? 2 : 1) && st == ATDCT16_OK; ++half) {
            bc.ctas_per_sm = half ? std::max(1, maxc / 2) : 0;
            float ms = 0.f;
            st = time_shape(b, best_cfg, sms * best_ctas, bc, stream, e0, e1, &ms);
            if (st != ATDCT16_OK) break;
            b->cands.push_back(tune_point(best_cfg, best_ctas, bc, ms));
            if (ms < best) {
              best = ms;
              best_box = bc;
            }
          }
        }
  }
  if (has_general && st == ATDCT16_OK) {
    const ZonalConfig gens[] = {{kZonalSwar, 4, 1}, {kZonalF32, 4, 1}, {kZonalMma, 4, 1}, {kZonalTc, 4, 1}};
    best = 1e30f;
    for (const ZonalConfig& c : gens) {
      const int maxc = zonal_config_max_ctas_per_sm(c);
      const int opts[2] = {maxc, std::max(1, maxc / 2)};
      for (int oi = 0; oi < (maxc > 1 ? 2 : 1) && st == ATDCT16_OK; ++oi) {
        float ms = 0.f;
        st = time_shape(b, c, sms * opts[oi], best_box, stream, e0, e1, &ms);
        if (st != ATDCT16_OK) break;
        b->cands.push_back(tune_point(c, opts[oi], best_box, ms, 1));
        if (ms < best) {
          best = ms;
          best_cfg = c;
          best_ctas = opts[oi];
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ATDCT16_OK) return st;
  b->cfg = best_cfg;
  b->ctas = best_ctas;
  b->box = best_box;
  b->tuned_ms = best;
  return ATDCT16_OK;
}

void free_batch(atdct16_batch_st* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_jobs);
  cudaFree(b->d_tile_sse);
  cudaFree(b->d_status);
  delete b;
}

}  // namespace

extern "C" {

atdct16_status atdct16_batch_create(atdct16_plan_t plan, const atdct16_image* h_images, int32_t n, double* d_psnr,
                                    double* d_sse, uint32_t flags, cudaStream_t stream, atdct16_batch_t* out) {
  if (!out) return ATDCT16_EINVAL;
  *out = nullptr;
  if (!plan || !h_images || !d_psnr || n < 1 ||
      (flags & ~(ATDCT16_BATCH_AUTOTUNE | ATDCT16_BATCH_GRAPH | ATDCT16_BATCH_VARIANT_MASK | ATDCT16_BATCH_SHAPE_MASK)))
    return ATDCT16_EINVAL;
  // a pinned box shape (fields: tiles per CTA code, depth, width code) excludes autotuning
  const unsigned shape = (flags & ATDCT16_BATCH_SHAPE_MASK) >> ATDCT16_BATCH_SHAPE_SHIFT;
  BoxConfig pinned_box = default_box_config();
  if (shape) {
    const unsigned wc = shape & 3u, d = (shape >> 2) & 3u, vc = (shape >> 4) & 3u;
    pinned_box = BoxConfig{wc == 1 ? 2 : (wc == 2 ? 4 : 8), (int)d, vc == 1 ? 8 : 16, 0};
    if ((flags & ATDCT16_BATCH_AUTOTUNE) || wc == 0 || vc == 0 || vc == 3 || !box_config_supported(pinned_box))
      return ATDCT16_EINVAL;
  }
  // a pinned kernel variant (1 + variant in the variant field) excludes autotuning
  const unsigned pinned = (flags & ATDCT16_BATCH_VARIANT_MASK) >> ATDCT16_BATCH_VARIANT_SHIFT;
  if (pinned && ((flags & ATDCT16_BATCH_AUTOTUNE) ||
                 !zonal_config_supported(ZonalConfig{(int)pinned - 1, kZonalWarps, 1})))
    return ATDCT16_EINVAL;
  for (int i = 0; i < n; ++i) {
    const atdct16_status s = check_zonal_image(h_images[i]);
    if (s != ATDCT16_OK) return s;
  }
  if ((flags & ATDCT16_BATCH_AUTOTUNE) && dst_overlaps_src(h_images, n)) return ATDCT16_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ATDCT16_ECUDA;
  if (dev != plan_device(plan)) return ATDCT16_EINVAL;

  std::vector<ImageJob> jobs(2 * (size_t)n);
  long long tiles = 0;
  for (int i = 0; i < n; ++i) {
    const atdct16_image& im = h_images[i];
    ImageJob& J = jobs[i];
    J.src = static_cast<const uint8_t*>(im.src);
    J.dst = static_cast<uint8_t*>(im.dst);
    J.src_pitch = im.src_pitch;
    J.dst_pitch = im.dst_pitch;
    J.width = im.width;
    J.height = im.height;
    J.tiles_x = (im.width + kTileW - 1) / kTileW;
    J.param = im.r_or_qp;
    J.tile_begin = tiles;
    J.level_base = 0;
    tiles += (long long)J.tiles_x * (im.height / kTileH);
  }

  atdct16_batch_st* b = new (std::nothrow) atdct16_batch_st();
  if (!b) return ATDCT16_ENOMEM;
  b->plan = plan;
  b->device = dev;
  b->n = n;
  b->ntiles = tiles;
  b->d_psnr = d_psnr;
  b->d_sse = d_sse;
  b->last_stream = stream;
  zonal_order(jobs.data(), n, jobs.data() + n, &b->split);
  cudaError_t e = cudaMalloc(&b->d_jobs, 2 * sizeof(ImageJob) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tile_sse, sizeof(float) * std::max<long long>(1, tiles));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_jobs, jobs.data(), 2 * sizeof(ImageJob) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    free_batch(b);
    return e == cudaErrorMemoryAllocation ? ATDCT16_ENOMEM : ATDCT16_ECUDA;
  }

  const int sms = plan_num_sms(plan);
  b->cfg = pinned ? ZonalConfig{(int)pinned - 1, kZonalWarps, 1} : default_zonal_config();
  b->ctas = zonal_config_max_ctas_per_sm(b->cfg);
  b->box = pinned_box;
  if (flags & ATDCT16_BATCH_AUTOTUNE) {
    const unsigned long long key = shape_key(h_images, n, sms);
    ZonalConfig c;
    BoxConfig bc;
    int ctas;
    float ms;
    if (plan_tune_lookup(plan, key, &c, &ctas, &bc, &ms) || file_lookup(key, &c, &ctas, &bc, &ms)) {
      b->cfg = c;
      b->ctas = ctas;
      b->box = bc;
      b->tuned_ms = ms;
      plan_tune_store(plan, key, c, ctas, bc, ms);
    } else {
      const atdct16_status s = autotune(b, sms, stream);
      if (s != ATDCT16_OK) {
        free_batch(b);
        return s;
      }
      plan_tune_store(plan, key, b->cfg, b->ctas, b->box, b->tuned_ms);
      file_store(key, b->cfg, b->ctas, b->box, b->tuned_ms);
    }
  }
  b->grid = grid_for(b->cfg, b->ctas, sms, tiles);
  b->cfg.test_stall = plan_test_stall_mma(plan) ? 1 : 0;

  if (flags & ATDCT16_BATCH_GRAPH) {
    // Capture on a private stream so that the caller's stream is untouched.
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      // launches with dynamic shared memory above 48 KB set their attribute
      // first; do one uncaptured launch so that happens outside the capture
      e = launch_batch_once(b, b->cfg, b->grid, b->box, cs);
      if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t le = launch_batch_once(b, b->cfg, b->grid, b->box, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (le != cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      cudaStreamDestroy(cs);
    }
    if (e != cudaSuccess) {
      free_batch(b);
      return ATDCT16_ECUDA;
    }
  }
  *out = b;
  return ATDCT16_OK;
}

atdct16_status atdct16_batch_launch(atdct16_batch_t b, cudaStream_t stream) {
  if (!b) return ATDCT16_EINVAL;
  b->last_stream = stream;
  cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, stream) : launch_batch_once(b, b->cfg, b->grid, b->box, stream);
  return e == cudaSuccess ? ATDCT16_OK : ATDCT16_ECUDA;
}

atdct16_status atdct16_batch_last_device_status(atdct16_batch_t b) {
  if (!b) return ATDCT16_EINVAL;
  if (b->last_stream && cudaStreamSynchronize(b->last_stream) != cudaSuccess) return ATDCT16_ECUDA;
  int v = 0;
  if (cudaMemcpy(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ATDCT16_ECUDA;
  return v == kDevOk ? ATDCT16_OK : (v == kDevTimeout ? ATDCT16_ETIMEOUT : ATDCT16_EDEVICE);
}

atdct16_status atdct16_batch_info(atdct16_batch_t b, int32_t* variant, int32_t* warps, int32_t* prefetch,
                                  int32_t* grid, int64_t* tiles, float* tuned_ms) {
  if (!b) return ATDCT16_EINVAL;
  if (variant) *variant = b->cfg.variant;
  if (warps) *warps = b->cfg.warps;
  if (prefetch) *prefetch = b->cfg.prefetch;
  if (grid) *grid = b->grid;
  if (tiles) *tiles = b->ntiles;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  return ATDCT16_OK;
}

atdct16_status atdct16_batch_tuning(atdct16_batch_t b, atdct16_tune_point* chosen, atdct16_tune_point* candidates,
                                    int32_t max_candidates, int32_t* n_candidates) {
  if (!b || max_candidates < 0 || (max_candidates > 0 && !candidates)) return ATDCT16_EINVAL;
  if (chosen) *chosen = tune_point(b->cfg, b->ctas, b->box, b->tuned_ms);
  const int n = (int)b->cands.size();
  for (int i = 0; i < n && i < max_candidates; ++i) candidates[i] = b->cands[i];
  if (n_candidates) *n_candidates = n;
  return ATDCT16_OK;
}

atdct16_status atdct16_batch_destroy(atdct16_batch_t b) {
  if (!b) return ATDCT16_EINVAL;
  cudaSetDevice(b->device);
  if (b->last_stream) cudaStreamSynchronize(b->last_stream);
  free_batch(b);
  return ATDCT16_OK;
}

}  // extern "C"
