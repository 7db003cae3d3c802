// Zonal compression entry point that allocates no memory.
//
// Some callers cannot allocate device memory when they compress: code that
// runs on a fixed memory budget reserved at start-up (embedded or
// safety-certified systems), latency-critical paths where cudaMalloc's
// implicit device synchronisation is not acceptable, and applications whose
// own allocator owns all device memory.  atdct16_compress_zonal_noalloc serves
// them: it needs no plan, and the only device memory it uses besides the
// caller's inputs and outputs is the file-scope scratch array below, which
// every GPU that loads the library holds until the process exits.
//
// The scratch holds the job descriptors (the table and its class-ordered
// copy that the kernels read), the zonal weight table, the per-tile partial
// sums and the device status word.  Every call shares it and it keeps
// the last call's contents; each call rewrites the descriptors, clears the
// status word and writes every partial it later reads.  Calls that overlap on
// the GPU (different streams, or several host threads) race on it.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "../../include/atdct16.h"
#include "atdct16_butterfly.cuh"
#include "atdct16_internal.h"
#include "atdct16_zigzag.cuh"

namespace atdct16 {
namespace {

constexpr int kNoAllocMaxImages = 64;
constexpr long long kNoAllocMaxTiles = 1 << 17;  // 131072 tiles of 16 x 128 pixels

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffJobs = 0;
constexpr size_t kOffStatus = align256(kOffJobs + 2 * sizeof(ImageJob) * kNoAllocMaxImages);
constexpr size_t kOffWtab = align256(kOffStatus + sizeof(int));
constexpr size_t kOffTiles = align256(kOffWtab + sizeof(float2) * kZonalTableEntries);
constexpr size_t kScratchBytes = align256(kOffTiles + sizeof(float) * kNoAllocMaxTiles);  // ~1.03 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Descriptors travel as a kernel parameter, so no host-to-device copy (and no
// staging allocation) is needed.
struct JobPack {
  ImageJob jobs[kNoAllocMaxImages];
};

// Copies n descriptors to slot `first` of the scratch's table; the first of
// a call's two copies also clears the status word.
__global__ void noalloc_stage_jobs(const __grid_constant__ JobPack pack, int n, int first, unsigned char* scratch) {
  ImageJob* jobs = reinterpret_cast<ImageJob*>(scratch + kOffJobs) + first;
  for (int i = threadIdx.x; i < n; i += blockDim.x) jobs[i] = pack.jobs[i];
  if (threadIdx.x == 0 && first == 0) *reinterpret_cast<int*>(scratch + kOffStatus) = kDevOk;
}

// Fills the zonal weight table (kw, dw) for every r in 0..256 from the
// zig-zag rank and the row non-zero counts of T: W = 48 / nnz, entries
// (keep, 1 - keep) * W_u * W_c / 256.
struct TableSeed {
  unsigned char rank[256];
  int nnz[16];
};

__global__ void noalloc_fill_weights(const __grid_constant__ TableSeed seed, unsigned char* scratch) {
  float2* wtab = reinterpret_cast<float2*>(scratch + kOffWtab);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kZonalTableEntries; i += gridDim.x * blockDim.x) {
    const int r = i >> 8, c = (i >> 4) & 15, u = i & 15;
    const float wgt = (48.0f / seed.nnz[u]) * (48.0f / seed.nnz[c]) * (1.0f / 256.0f);
    const bool keep = seed.rank[u * 16 + c] < r;
    wtab[i] = make_float2(keep ? wgt : 0.f, keep ? 0.f : wgt);
  }
}

struct DeviceSetup {
  std::atomic<bool> ready{false};
  unsigned char* ptr = nullptr;
  int grid = 0;
  int sms = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: look up the device address of
// the scratch array and fill its weight table.
atdct16_status setup_device(int dev, cudaStream_t stream, DeviceSetup** out) {
  if (dev < 0 || dev >= kMaxDevices) return ATDCT16_EUNSUPPORTED;
  DeviceSetup& s = g_setup[dev];
  if (!s.ready.load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!s.ready.load(std::memory_order_relaxed)) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ATDCT16_ECUDA;
      int sms = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ATDCT16_ECUDA;
      // Stream capture would record the table fill instead of running it, and
      // the synchronisation below would then fail: refuse before enqueuing.
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return ATDCT16_ECUDA;
      if (cap != cudaStreamCaptureStatusNone) return ATDCT16_EUNSUPPORTED;
      TableSeed seed;
      for (int w = 0; w < 256; ++w) seed.rank[w] = (unsigned char)zigzag_rank(w);  // Sec. 4 scan
      row_nonzeros(seed.nnz);
      noalloc_fill_weights<<<64, 256, 0, stream>>>(seed, static_cast<unsigned char*>(p));
      // later calls may come on other streams: the table must be complete
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess) return ATDCT16_ECUDA;
      s.ptr = static_cast<unsigned char*>(p);
      s.grid = sms * zonal_ctas_per_sm();
      s.sms = sms;
      s.ready.store(true, std::memory_order_release);
    }
  }
  *out = &s;
  return ATDCT16_OK;
}

}  // namespace
}  // namespace atdct16

using namespace atdct16;

extern "C" atdct16_status atdct16_noalloc_last_device_status(cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ATDCT16_ECUDA;
  if (dev < 0 || dev >= kMaxDevices || !g_setup[dev].ready.load(std::memory_order_acquire)) return ATDCT16_EINVAL;
  int v = 0;
  if (cudaMemcpyFromSymbolAsync(&v, g_noalloc_scratch, sizeof(int), kOffStatus, cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return ATDCT16_ECUDA;
  return v == kDevOk ? ATDCT16_OK : (v == kDevTimeout ? ATDCT16_ETIMEOUT : ATDCT16_EDEVICE);
}

extern "C" atdct16_status atdct16_compress_zonal_noalloc(const atdct16_image* h_images, int32_t n, double* d_psnr,
                                                         double* d_sse, cudaStream_t stream) {
  if (!h_images || !d_psnr || n < 1) return ATDCT16_EINVAL;
  if (n > kNoAllocMaxImages) return ATDCT16_ENOMEM;
  JobPack pack;
  std::memset(&pack, 0, sizeof(pack));
  long long tiles = 0;
  for (int i = 0; i < n; ++i) {
    const atdct16_image& im = h_images[i];
    if (!im.src || !im.dst || im.width <= 0 || im.height <= 0 || (im.width & 15) || (im.height & 15) ||
        im.src_pitch < im.width || im.dst_pitch < im.width || (im.src_pitch & 15) || (im.dst_pitch & 15) ||
        (reinterpret_cast<uintptr_t>(im.src) & 15) || (reinterpret_cast<uintptr_t>(im.dst) & 15) ||
        im.reserved != 0 || im.r_or_qp < 0 || im.r_or_qp > 256 || im.src_pitch >= ((int64_t)1 << 31) ||
        im.dst_pitch >= ((int64_t)1 << 31))
      return ATDCT16_EINVAL;
    ImageJob& J = pack.jobs[i];
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
  if (tiles > kNoAllocMaxTiles) return ATDCT16_ENOMEM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ATDCT16_ECUDA;
  DeviceSetup* s = nullptr;
  atdct16_status st = setup_device(dev, stream, &s);
  if (st != ATDCT16_OK) return st;
  unsigned char* p = s->ptr;
  JobPack ordered;
  std::memset(&ordered, 0, sizeof(ordered));
  ZonalSplit split;
  zonal_order(pack.jobs, n, ordered.jobs, &split);
  noalloc_stage_jobs<<<1, 64, 0, stream>>>(pack, n, 0, p);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    noalloc_stage_jobs<<<1, 64, 0, stream>>>(ordered, n, kNoAllocMaxImages, p);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return ATDCT16_ECUDA;
  const ImageJob* jobs = reinterpret_cast<const ImageJob*>(p + kOffJobs);
  e = launch_zonal_ordered(jobs + kNoAllocMaxImages, split, default_zonal_config(), s->grid, default_box_config(),
                           reinterpret_cast<const float2*>(p + kOffWtab), reinterpret_cast<float*>(p + kOffTiles),
                           reinterpret_cast<int*>(p + kOffStatus), s->sms, stream);
  if (e == cudaSuccess)
    e = launch_psnr_finalize(jobs, n, tiles, reinterpret_cast<const float*>(p + kOffTiles), 255.0, d_psnr, d_sse,
                             stream);
  return e == cudaSuccess ? ATDCT16_OK : ATDCT16_ECUDA;
}
