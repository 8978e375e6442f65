// Allocation-free batched polynomial encode.
//
// Some callers cannot allocate device memory at the moment they need to
// encode: allocator and memory-pool callbacks (for example a caching
// allocator that encodes the blocks it evicts) must not re-enter the
// allocator they are part of; embedders that reserve the whole device
// memory budget at start-up forbid allocations afterwards; and code on a
// latency-critical path cannot afford cudaMalloc / cudaFree, which may
// synchronise the device.  rs_init and rs_batch_create allocate (a status
// word, descriptor tables), so those callers get this entry point instead:
// every piece of scratch the batched kernel needs -- its descriptor tables
// and pointer table, and a status word -- lives in one file-scope static
// device array of fixed size, and the tables reach it through small upload
// kernels whose parameters carry them by value (no host staging buffer, no
// copy from pageable memory).  The caller passes only the data and parity
// blocks (and, if it wants wait timeouts reported, an int of its own).
//
// The array is shared by every call on a device and keeps the last call's
// contents: each call clears the status word and rewrites the tables before
// its encode kernel runs.  Calls whose work overlaps on the GPU (different
// streams without ordering) race on the array: order them on one stream or
// synchronise between them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "launch.hpp"
#include "registry.hpp"
#include "rs_gb300.h"

namespace {

constexpr size_t kScratchBytes = 256u * 1024u;   // per device, reserved at module load
constexpr size_t kStatusBytes = 256;             // status word, padded
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// One upload: `bytes` (a multiple of 16) bytes of table image written at
// byte `dst` of the static array.  Passed by value as the kernel's
// parameter, so nothing on the host has to outlive the call.
constexpr uint32_t kUploadBytes = 8192;
struct UploadChunk {
  uint32_t dst;
  uint32_t bytes;
  uint32_t pad[2];
  uint4 data[kUploadBytes / 16];
};
static_assert(sizeof(UploadChunk) <= 32000, "kernel parameter space");

__global__ void __launch_bounds__(256) rs_noalloc_upload(const __grid_constant__ UploadChunk c) {
  uint4* dst = reinterpret_cast<uint4*>(g_noalloc_scratch + c.dst);
  for (uint32_t i = threadIdx.x; i < c.bytes / 16u; i += blockDim.x) dst[i] = c.data[i];
}

static std::once_flag g_setup_once[kMaxDevices];
static cudaError_t g_setup_err[kMaxDevices];
static unsigned char* g_scratch_dev[kMaxDevices];

rs_status fail_na(rs_status s, const std::string& msg) {
  rsgb::set_last_error(msg);
  return s;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte offsets of the tables in the array for `used` stripes of n blocks.
struct Layout {
  size_t descs, ptrs, end;
};
Layout layout_for(size_t used, int n_blocks) {
  Layout l;
  l.descs = kStatusBytes;
  l.ptrs = l.descs + align_up(sizeof(rsgb::StripeDesc) * used, 256);
  l.end = align_up(l.ptrs + sizeof(uint64_t) * used * (size_t)n_blocks, 16);
  return l;
}

// Streams the table image into the array, one upload kernel per
// kUploadBytes, in order; bytes are appended at consecutive offsets.
class Uploader {
 public:
  Uploader(cudaStream_t st) : st_(st) { reset(0); }
  void put(const void* src, size_t n) {
    const unsigned char* s = static_cast<const unsigned char*>(src);
    while (n && err_ == cudaSuccess) {
      const size_t take = std::min(n, (size_t)kUploadBytes - fill_);
      memcpy(reinterpret_cast<unsigned char*>(c_.data) + fill_, s, take);
      fill_ += take;
      s += take;
      n -= take;
      if (fill_ == kUploadBytes) flush();
    }
  }
  void zeros(size_t n) {
    static const unsigned char z[256] = {};
    while (n) {
      const size_t take = std::min(n, sizeof(z));
      put(z, take);
      n -= take;
    }
  }
  cudaError_t finish() {
    if (fill_) {
      const size_t pad = align_up(fill_, 16) - fill_;
      memset(reinterpret_cast<unsigned char*>(c_.data) + fill_, 0, pad);
      fill_ += pad;
      flush();
    }
    return err_;
  }
  size_t offset() const { return base_ + fill_; }

 private:
  void reset(size_t base) {
    base_ = base;
    fill_ = 0;
  }
  void flush() {
    c_.dst = (uint32_t)base_;
    c_.bytes = (uint32_t)fill_;
    rs_noalloc_upload<<<1, 256, 0, st_>>>(c_);
    if (err_ == cudaSuccess) err_ = cudaGetLastError();
    reset(base_ + fill_);
  }
  cudaStream_t st_;
  UploadChunk c_;
  size_t base_ = 0, fill_ = 0;
  cudaError_t err_ = cudaSuccess;
};

}  // namespace

extern "C" rs_status rs_poly_encode_stripes_noalloc(int k, int m, int w, int n_stripes,
                                                     const void* const* data_ptrs, void* const* parity_ptrs,
                                                     const size_t* block_bytes, int* device_status,
                                                     void* stream) {
  using namespace rsgb;
  if (w != 8 && w != 16) return fail_na(RS_EINVAL, "w must be 8 or 16");
  if (k < 1 || m < 1) return fail_na(RS_EINVAL, "need k >= 1 and m >= 1");
  if ((long)k + m > (1L << w) - 1) return fail_na(RS_EINVAL, "k + m must be <= 2^w - 1");
  if (m > kMaxM || k + m > kMaxBlocks || (w == 16 && m > 4))
    return fail_na(RS_EUNSUPPORTED, "device path limits: m <= 8 (m <= 4 for w = 16), k + m <= 64");
  if (n_stripes < 0) return fail_na(RS_EINVAL, "negative stripe count");
  if (n_stripes == 0) {
    rsgb::clear_last_error();
    return RS_OK;
  }
  if (!data_ptrs || !parity_ptrs || !block_bytes) return fail_na(RS_EINVAL, "null argument array");
  if (device_status && ((uintptr_t)device_status & 3u))
    return fail_na(RS_EINVAL, "device_status must be 4-byte aligned");
  const int n = k + m;
  // per-stripe argument checks (same rules as rs_encode)
  size_t used = 0;
  for (int s = 0; s < n_stripes; ++s) {
    const size_t B = block_bytes[s];
    if (B == 0) continue;
    ++used;
    if (w == 16 && (B & 1u)) return fail_na(RS_EINVAL, "block_bytes must be even for w = 16");
    if (B > ((size_t)1 << 40)) return fail_na(RS_EINVAL, "block_bytes too large");
    uintptr_t p[kMaxBlocks];
    for (int i = 0; i < k; ++i) p[i] = (uintptr_t)data_ptrs[(size_t)s * k + i];
    for (int j = 0; j < m; ++j) p[k + j] = (uintptr_t)parity_ptrs[(size_t)s * m + j];
    for (int i = 0; i < n; ++i) {
      if (!p[i]) return fail_na(RS_EINVAL, "stripe " + std::to_string(s) + ": null block pointer");
      if (p[i] & 15u) return fail_na(RS_EINVAL, "stripe " + std::to_string(s) + ": block pointers must be 16-byte aligned");
    }
    std::sort(p, p + n);
    for (int i = 1; i < n; ++i)
      if (p[i] - p[i - 1] < B) return fail_na(RS_EINVAL, "stripe " + std::to_string(s) + ": blocks overlap");
  }
  if (used == 0) {
    rsgb::clear_last_error();
    return RS_OK;
  }
  const Layout lay = layout_for(used, n);
  if (lay.end > kScratchBytes)
    return fail_na(RS_EINVAL, "request needs " + std::to_string(lay.end) + " bytes of scratch; the fixed array holds " +
                                  std::to_string(kScratchBytes) + " bytes (" + std::to_string(used) +
                                  " non-empty stripes of " + std::to_string(n) + " blocks)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(RS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(RS_EUNSUPPORTED, "device index out of range");
  // One-time set-up per device, with that device current: the device address
  // of the static array (in host code its name is only a stand-in).
  std::call_once(g_setup_once[dev], [&] {
    void* ptr = nullptr;
    g_setup_err[dev] = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    g_scratch_dev[dev] = static_cast<unsigned char*>(ptr);
  });
  if (g_setup_err[dev] != cudaSuccess || !g_scratch_dev[dev])
    return fail_na(RS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(g_setup_err[dev]));
  unsigned char* scratch = g_scratch_dev[dev];

  KernelKey key;
  key.family = kFamPoly;
  key.w = w;
  key.m = m;
  key.op = kOpEncode;
  const KernelEntry* entry = find_kernel(key);
  if (!entry) return fail_na(RS_EUNSUPPORTED, "no kernel compiled for this code");
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail_na(RS_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));

  TuneCfg tune;
  int nc = std::max(1, std::min(tune.consumer_warps, entry->max_warps));
  if (entry->producer_warps == 4) nc = std::max(4, nc / 4 * 4);
  const uint32_t slice = (uint32_t)(nc * entry->groups) * segment_bytes(w);
  uint32_t depth = (uint32_t)tune.depth;
  while (depth > 2 && ring_smem_bytes(depth, slice) > kMaxDynamicSmem) --depth;
  // tile numbering of the launch (32-bit in the kernel)
  uint64_t tiles = 0;
  for (int s = 0; s < n_stripes; ++s) tiles += (block_bytes[s] + slice - 1) / slice;
  if (tiles > 0xFFFFFFFFull) return fail_na(RS_EINVAL, "too many tiles in one call (more than 2^32)");

  cudaStream_t st = (cudaStream_t)stream;
  Uploader up(st);
  up.zeros(kStatusBytes);  // the status word starts at zero
  uint32_t t = 0, np = 0;
  for (int s = 0; s < n_stripes; ++s) {
    const size_t B = block_bytes[s];
    if (B == 0) continue;
    StripeDesc d;
    memset(&d, 0, sizeof(d));
    d.bytes = B;
    d.tile_begin = t;
    d.ptr_off = np;
    d.n_in = (uint16_t)k;
    d.n_out = (uint16_t)m;
    d.op = kOpEncode;
    d.m = (uint8_t)m;
    d.k = (uint8_t)k;
    d.layout = kLayoutSymbol;
    up.put(&d, sizeof(d));
    t += (uint32_t)((B + slice - 1) / slice);
    np += (uint32_t)n;
  }
  up.zeros(lay.ptrs - up.offset());
  for (int s = 0; s < n_stripes; ++s) {
    if (block_bytes[s] == 0) continue;
    // LFSR consumption order: d_{k-1} first (§3.2 Eq. 2), then the outputs
    for (int i = k - 1; i >= 0; --i) {
      const uint64_t v = (uint64_t)(uintptr_t)data_ptrs[(size_t)s * k + i];
      up.put(&v, sizeof(v));
    }
    for (int j = 0; j < m; ++j) {
      const uint64_t v = (uint64_t)(uintptr_t)parity_ptrs[(size_t)s * m + j];
      up.put(&v, sizeof(v));
    }
  }
  e = up.finish();
  if (e != cudaSuccess) return fail_na(RS_ECUDA, std::string("scratch upload: ") + cudaGetErrorString(e));

  JobParams p;
  memset(&p, 0, sizeof(p));
  p.stripes = reinterpret_cast<const StripeDesc*>(scratch + lay.descs);
  p.ptrs = reinterpret_cast<const uint64_t*>(scratch + lay.ptrs);
  p.coef = nullptr;
  p.status = device_status ? device_status : reinterpret_cast<int*>(scratch);
  p.counts = nullptr;
  p.n_stripes = (uint32_t)used;
  p.total_tiles = (uint32_t)tiles;
  p.slice_bytes = slice;
  p.depth = depth;
  LaunchShape sh;
  sh.threads = (nc + entry->producer_warps) * 32;
  sh.smem = ring_smem_bytes(depth, slice);
  sh.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)sms));
  e = entry->launch(p, sh, st);
  if (e != cudaSuccess) return fail_na(RS_ECUDA, std::string(entry->name) + ": " + cudaGetErrorString(e));
  rsgb::clear_last_error();
  return RS_OK;
}
