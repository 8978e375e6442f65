// Batched block transfer: many byte ranges copied by one kernel launch.
//
// Moving the blocks of a batch between host and device with one copy call
// per block costs a host-side call (several microseconds) per block; with
// hundreds of blocks per batch the host thread, not the link, becomes the
// limit.  On a system with unified addressing every pinned host allocation
// is mapped into the device address space, so a kernel can read and write
// it directly at the host link's bandwidth.  rs_copy_blocks hands the small
// ranges of a batch to such a kernel (one launch per kMaxRuns ranges,
// descriptors passed as kernel parameters: no device allocation, capturable
// in a graph) and gives each large range to the copy engines with one
// cudaMemcpyAsync, issued from here at a small fraction of the cost of a
// call from Python; the copy engines use no SMs, so large transfers do not
// take SM slots from the coding kernels running beside them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <string>

#include "launch.hpp"
#include "rs_gb300.h"

namespace {

constexpr int kMaxRuns = 512;                 // ranges per launch (parameter space)
constexpr uint32_t kChunk = 32u * 1024u;      // bytes per warp work item
constexpr int kThreads = 256;
constexpr size_t kEngineBytes = 4u << 20;  // default: ranges at least this large go to the copy engines

struct CopyParams {
  uint64_t src[kMaxRuns];
  uint64_t dst[kMaxRuns];
  uint64_t bytes[kMaxRuns];
  uint32_t chunk_begin[kMaxRuns + 1];  // prefix sums of the ranges' chunk counts
  int n;
};
static_assert(sizeof(CopyParams) <= 32000, "kernel parameter space");
// Per-range limit (256 GiB) such that the chunk count of kMaxRuns ranges fits
// the 32-bit prefix sums.
constexpr uint64_t kMaxRangeBytes = (uint64_t)kChunk * 0x7FFFFFu;
static_assert((uint64_t)kMaxRuns * 0x7FFFFFu <= 0xFFFFFFFFull, "prefix sums fit 32 bits");

__global__ void __launch_bounds__(kThreads) rs_copy_kernel(const __grid_constant__ CopyParams p) {
  const uint32_t warps = blockDim.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t total = p.chunk_begin[p.n];
  for (uint32_t item = blockIdx.x * warps + (threadIdx.x >> 5); item < total; item += gridDim.x * warps) {
    // range r holds chunk items [chunk_begin[r], chunk_begin[r + 1])
    int lo = 0, hi = p.n;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (p.chunk_begin[mid] <= item) lo = mid;
      else hi = mid;
    }
    const uint64_t off = (uint64_t)(item - p.chunk_begin[lo]) * kChunk;
    const uint64_t len = min((uint64_t)kChunk, p.bytes[lo] - off);
    const uint8_t* s = reinterpret_cast<const uint8_t*>(p.src[lo]) + off;
    uint8_t* d = reinterpret_cast<uint8_t*>(p.dst[lo]) + off;
    const uint64_t len16 = len & ~15ull;
    // four 16-byte loads in flight per lane before the stores
    uint64_t o = (uint64_t)lane * 16u;
    for (; o + 3u * 512u + 16u <= len16; o += 4u * 512u) {
      const uint4 a = *reinterpret_cast<const uint4*>(s + o);
      const uint4 b = *reinterpret_cast<const uint4*>(s + o + 512u);
      const uint4 c = *reinterpret_cast<const uint4*>(s + o + 1024u);
      const uint4 e = *reinterpret_cast<const uint4*>(s + o + 1536u);
      *reinterpret_cast<uint4*>(d + o) = a;
      *reinterpret_cast<uint4*>(d + o + 512u) = b;
      *reinterpret_cast<uint4*>(d + o + 1024u) = c;
      *reinterpret_cast<uint4*>(d + o + 1536u) = e;
    }
    for (; o + 16u <= len16; o += 512u) *reinterpret_cast<uint4*>(d + o) = *reinterpret_cast<const uint4*>(s + o);
    for (uint64_t t = len16 + lane; t < len; t += 32u) d[t] = s[t];
  }
}

}  // namespace

extern "C" rs_status rs_copy_blocks(void* const* dst, const void* const* src, const size_t* bytes, int n,
                                    size_t engine_min_bytes, void* stream) {
  using namespace rsgb;
  clear_last_error();
  if (n < 0 || (n > 0 && (!dst || !src || !bytes))) {
    set_last_error("rs_copy_blocks: n < 0 or null array");
    return RS_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    if (bytes[i] && (!dst[i] || !src[i])) {
      set_last_error("rs_copy_blocks: null pointer in range " + std::to_string(i));
      return RS_EINVAL;
    }
    if ((reinterpret_cast<uintptr_t>(dst[i]) | reinterpret_cast<uintptr_t>(src[i])) & 15u) {
      set_last_error("rs_copy_blocks: range " + std::to_string(i) + " is not 16-byte aligned");
      return RS_EINVAL;
    }
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(src[i]), d0 = reinterpret_cast<uintptr_t>(dst[i]);
    if (bytes[i] && s0 < d0 + bytes[i] && d0 < s0 + bytes[i]) {
      set_last_error("rs_copy_blocks: range " + std::to_string(i) + " overlaps itself");
      return RS_EINVAL;
    }
    if (bytes[i] > kMaxRangeBytes) {
      set_last_error("rs_copy_blocks: range " + std::to_string(i) + " is too large");
      return RS_EINVAL;
    }
    // Only device memory and page-locked host memory are addressable by the
    // kernel: check the first and the last byte of both ends of the range.
    if (bytes[i]) {
      const void* ends[4] = {src[i], static_cast<const uint8_t*>(src[i]) + bytes[i] - 1, dst[i],
                             static_cast<const uint8_t*>(dst[i]) + bytes[i] - 1};
      for (const void* q : ends) {
        cudaPointerAttributes a;
        const cudaError_t pe = cudaPointerGetAttributes(&a, q);
        if (pe != cudaSuccess || a.type == cudaMemoryTypeUnregistered || !a.devicePointer) {
          cudaGetLastError();  // clear the error the query may have recorded
          set_last_error("rs_copy_blocks: range " + std::to_string(i) +
                         " is not device memory or page-locked host memory");
          return RS_EINVAL;
        }
      }
    }
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_last_error(std::string("rs_copy_blocks: ") + cudaGetErrorString(e));
    return RS_ECUDA;
  }
  CopyParams* p = new (std::nothrow) CopyParams();
  if (!p) {
    set_last_error("rs_copy_blocks: out of host memory");
    return RS_ENOMEM;
  }
  rs_status status = RS_OK;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t engine_min = engine_min_bytes ? engine_min_bytes : kEngineBytes;
  auto flush = [&]() {
    if (p->n == 0) return;
    const uint32_t items = p->chunk_begin[p->n];
    if (items) {
      const uint32_t want = (items + kThreads / 32 - 1) / (kThreads / 32);
      const int grid = (int)std::max<uint32_t>(1, std::min<uint32_t>(want, (uint32_t)sms));
      rs_copy_kernel<<<grid, kThreads, 0, st>>>(*p);
      const cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) {
        set_last_error(std::string("rs_copy_blocks: ") + cudaGetErrorString(le));
        status = RS_ECUDA;
      }
    }
    p->n = 0;
  };
  p->n = 0;
  p->chunk_begin[0] = 0;
  for (int i = 0; i < n && status == RS_OK; ++i) {
    if (!bytes[i]) continue;
    if (bytes[i] >= engine_min) {
      e = cudaMemcpyAsync(dst[i], src[i], bytes[i], cudaMemcpyDefault, st);
      if (e != cudaSuccess) {
        set_last_error(std::string("rs_copy_blocks: ") + cudaGetErrorString(e));
        status = RS_ECUDA;
      }
      continue;
    }
    const int j = p->n;
    p->src[j] = reinterpret_cast<uint64_t>(src[i]);
    p->dst[j] = reinterpret_cast<uint64_t>(dst[i]);
    p->bytes[j] = bytes[i];
    p->chunk_begin[j + 1] = p->chunk_begin[j] + (uint32_t)((bytes[i] + kChunk - 1) / kChunk);
    if (++p->n == kMaxRuns) flush();
  }
  if (status == RS_OK) flush();
  delete p;
  return status;
}
