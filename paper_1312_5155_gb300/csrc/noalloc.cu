// Allocation-free batched polynomial encode.
//
// Some callers cannot allocate device memory at the time they need to encode:
// code running while a CUDA stream is being captured into a graph (where
// cudaMalloc is not allowed), allocator callbacks and memory-pool hooks that
// must not re-enter the allocator, and embedders that own the whole device
// memory budget and forbid allocations after start-up.  rs_init / rs_batch_*
// allocate (a status word, descriptor tables), so those callers get this
// entry point instead: it keeps every piece of scratch the batched kernel
// needs -- its descriptor tables, pointer table and status word -- in one
// file-scope static device array of fixed size.  The caller passes only the
// data and parity blocks.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the status word is cleared at the start of every call and the
// tables are rewritten.  Calls whose work overlaps on the GPU (different
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

constexpr size_t kScratchBytes = 256u * 1024u;   // per device, allocated at module load
constexpr size_t kStatusBytes = 256;             // status word, padded
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host-side image of the tables, copied into the device array per call.
static unsigned char g_stage[kScratchBytes];
static std::mutex g_stage_mu;

static std::once_flag g_setup_once[kMaxDevices];
static cudaError_t g_setup_err[kMaxDevices];
static unsigned char* g_scratch_dev[kMaxDevices];

rs_status fail_na(rs_status s, const std::string& msg) {
  rsgb::set_last_error(msg);
  return s;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes of scratch a call with n stripes of n_blocks pointers needs.
size_t scratch_needed(int n_stripes, int n_blocks) {
  return kStatusBytes + align_up(sizeof(rsgb::StripeDesc) * (size_t)n_stripes, 256) +
         sizeof(uint64_t) * (size_t)n_stripes * (size_t)n_blocks;
}

}  // namespace

extern "C" rs_status rs_poly_encode_stripes_noalloc(int k, int m, int w, int n_stripes,
                                                     const void* const* data_ptrs, void* const* parity_ptrs,
                                                     const size_t* block_bytes, void* stream) {
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
  const int n = k + m;
  const size_t need = scratch_needed(n_stripes, n);
  if (need > kScratchBytes)
    return fail_na(RS_EINVAL, "request needs " + std::to_string(need) + " bytes of scratch; the fixed array holds " +
                                  std::to_string(kScratchBytes) + " bytes (" + std::to_string(n_stripes) +
                                  " stripes of " + std::to_string(n) + " blocks)");
  // per-stripe argument checks (same rules as rs_encode)
  for (int s = 0; s < n_stripes; ++s) {
    const size_t B = block_bytes[s];
    if (B == 0) continue;
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

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(RS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(RS_EUNSUPPORTED, "device index out of range");
  // One-time set-up per device, with that device current: the device address
  // of the static array (the host-side symbol is only a stand-in).
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
  const int nc = std::max(1, std::min(tune.consumer_warps, entry->max_warps));
  const uint32_t slice = (uint32_t)(nc * entry->groups) * segment_bytes(w);
  uint32_t depth = (uint32_t)tune.depth;
  while (depth > 2 && ring_smem_bytes(depth, slice) > kMaxDynamicSmem) --depth;

  std::lock_guard<std::mutex> lock(g_stage_mu);
  StripeDesc* descs = reinterpret_cast<StripeDesc*>(g_stage + kStatusBytes);
  const size_t ptr_off_bytes = kStatusBytes + align_up(sizeof(StripeDesc) * (size_t)n_stripes, 256);
  uint64_t* ptrs = reinterpret_cast<uint64_t*>(g_stage + ptr_off_bytes);
  uint32_t tiles = 0, used = 0, np = 0;
  for (int s = 0; s < n_stripes; ++s) {
    const size_t B = block_bytes[s];
    if (B == 0) continue;
    StripeDesc d;
    memset(&d, 0, sizeof(d));
    d.bytes = B;
    d.tile_begin = tiles;
    d.ptr_off = np;
    d.n_in = (uint16_t)k;
    d.n_out = (uint16_t)m;
    d.op = kOpEncode;
    d.m = (uint8_t)m;
    d.k = (uint8_t)k;
    d.layout = kLayoutSymbol;
    descs[used++] = d;
    tiles += (uint32_t)((B + slice - 1) / slice);
    // LFSR consumption order: d_{k-1} first (§3.2 Eq. 2), then the outputs
    for (int i = k - 1; i >= 0; --i) ptrs[np++] = (uint64_t)(uintptr_t)data_ptrs[(size_t)s * k + i];
    for (int j = 0; j < m; ++j) ptrs[np++] = (uint64_t)(uintptr_t)parity_ptrs[(size_t)s * m + j];
  }
  if (used == 0) {
    rsgb::clear_last_error();
    return RS_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // clear what must start at zero (the status word), then the tables
  e = cudaMemsetAsync(scratch, 0, kStatusBytes, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(scratch + kStatusBytes, g_stage + kStatusBytes,
                        ptr_off_bytes - kStatusBytes + sizeof(uint64_t) * np, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail_na(RS_ECUDA, std::string("scratch upload: ") + cudaGetErrorString(e));

  JobParams p;
  memset(&p, 0, sizeof(p));
  p.stripes = reinterpret_cast<const StripeDesc*>(scratch + kStatusBytes);
  p.ptrs = reinterpret_cast<const uint64_t*>(scratch + ptr_off_bytes);
  p.coef = nullptr;
  p.status = reinterpret_cast<int*>(scratch);
  p.counts = nullptr;
  p.n_stripes = used;
  p.total_tiles = tiles;
  p.slice_bytes = slice;
  p.depth = depth;
  LaunchShape sh;
  sh.threads = (nc + 1) * 32;
  sh.smem = ring_smem_bytes(depth, slice);
  sh.grid = (int)std::max<uint32_t>(1, std::min<uint32_t>(tiles, (uint32_t)sms));
  e = entry->launch(p, sh, st);
  if (e != cudaSuccess) return fail_na(RS_ECUDA, std::string(entry->name) + ": " + cudaGetErrorString(e));
  rsgb::clear_last_error();
  return RS_OK;
}
