// C ABI of the library (declared in include/rs_gb300.h): argument checks,
// per-code generator construction, decode-plan cache and kernel launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "launch.hpp"
#include "plan.hpp"
#include "rs_gb300.h"

using namespace rsgb;

namespace {

thread_local std::string g_last_error;

rs_status fail(rs_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

rs_status ok() {
  g_last_error.clear();
  return RS_OK;
}

rs_status cuda_fail(cudaError_t e, const char* what) {
  return fail(RS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

struct rs_code {
  int k = 0, m = 0, w = 0;
  Realization real = Realization::Poly;
  size_t packet_bytes = 2048;
  int read_mode = RS_READ_MIN;
  TuneCfg tune;
  std::vector<uint32_t> P;  // parity rows of the generator (matrix realizations)
  int device = 0;
  int num_sms = 0;
  int* d_status = nullptr;
  std::mutex mu;
  std::map<std::vector<int>, DecodePlan> plans;  // key: read mode, erasure list
};

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

rs_status check_device(const rs_code* c) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != c->device)
    return fail(RS_EINVAL, "code was created on device " + std::to_string(c->device) +
                               " but device " + std::to_string(dev) + " is current");
  return RS_OK;
}

// Blocks of one call must be pairwise disjoint (inputs are read while
// outputs are written).
bool disjoint(const std::vector<const void*>& ptrs, size_t bytes) {
  std::vector<uintptr_t> a;
  a.reserve(ptrs.size());
  for (auto p : ptrs) a.push_back((uintptr_t)p);
  std::sort(a.begin(), a.end());
  for (size_t i = 1; i < a.size(); ++i)
    if (a[i] - a[i - 1] < bytes) return false;
  return true;
}

rs_status check_blocks(const rs_code* c, const std::vector<const void*>& ptrs, size_t bytes) {
  for (size_t i = 0; i < ptrs.size(); ++i) {
    if (!ptrs[i]) return fail(RS_EINVAL, "null block pointer");
    if (!aligned16(ptrs[i])) return fail(RS_EINVAL, "block pointers must be 16-byte aligned");
  }
  if (c->w == 16 && (bytes & 1u)) return fail(RS_EINVAL, "block_bytes must be even for w = 16");
  if (c->real == Realization::Cauchy && bytes % ((size_t)c->w * c->packet_bytes))
    return fail(RS_EINVAL, "block_bytes must be a multiple of w * packet_bytes for the Cauchy realization");
  if (!disjoint(ptrs, bytes)) return fail(RS_EINVAL, "blocks of one call must not overlap");
  return RS_OK;
}

void fill_masks(uint32_t* dst, const DecodePlan& pl, int w) {
  const int M = pl.M;
  for (int t = 0; t < M; ++t)
    for (int j = 0; j < M; ++j)
      for (int c = 0; c < w; ++c)
        dst[(t * M + j) * w + c] = (t < pl.e && ((pl.W[t][j] >> c) & 1u)) ? 0xFFFFFFFFu : 0u;
}

// Shape of a launch over `total_tiles` tiles for a kernel with a consumer-warp cap.
LaunchShape make_shape(const rs_code* c, int warp_cap, uint32_t total_tiles, uint32_t& slice,
                       uint32_t& depth) {
  const int nc = std::max(1, std::min(c->tune.consumer_warps, warp_cap));
  slice = (uint32_t)nc * segment_bytes(c->w);
  depth = (uint32_t)std::max(2, c->tune.depth);
  while (depth > 2 && ring_smem_bytes(depth, slice) > kMaxDynamicSmem / (size_t)c->tune.ctas_per_sm) --depth;
  LaunchShape sh;
  sh.threads = (nc + 1) * 32;
  sh.smem = ring_smem_bytes(depth, slice);
  const uint32_t cap = (uint32_t)(c->num_sms * c->tune.ctas_per_sm);
  sh.grid = (int)std::max<uint32_t>(1, std::min(total_tiles, cap));
  return sh;
}

rs_status get_plan(rs_code* c, const int* er, int e, const DecodePlan** out) {
  std::vector<int> key;
  key.push_back(c->read_mode);
  key.insert(key.end(), er, er + e);
  std::lock_guard<std::mutex> g(c->mu);
  auto it = c->plans.find(key);
  if (it == c->plans.end()) {
    DecodePlan pl;
    std::string err;
    bool okp;
    if (c->real == Realization::Poly)
      okp = make_poly_decode_plan(c->k, c->m, c->w, er, e, c->read_mode == RS_READ_ALL, pl, err);
    else
      okp = make_matrix_decode_plan(c->k, c->m, c->w, c->P, er, e, c->read_mode == RS_READ_ALL, pl, err);
    if (!okp) return fail(e > c->m ? RS_ETOOMANY_ERASURES : RS_EINVAL, err);
    if (c->plans.size() > 4096) c->plans.clear();
    it = c->plans.emplace(key, pl).first;
  }
  *out = &it->second;
  return RS_OK;
}

}  // namespace

extern "C" {

int rs_version(void) { return 100; }

const char* rs_last_error(void) { return g_last_error.c_str(); }

rs_status rs_init(int k, int m, int w, int realization, rs_code** out) {
  if (!out) return fail(RS_EINVAL, "out is null");
  *out = nullptr;
  if (w != 8 && w != 16) return fail(RS_EINVAL, "w must be 8 or 16");
  if (k < 1 || m < 1) return fail(RS_EINVAL, "need k >= 1 and m >= 1");
  if (realization < RS_POLY || realization > RS_CAUCHY) return fail(RS_EINVAL, "unknown realization");
  if ((long)k + m > (1L << w) - 1) return fail(RS_EINVAL, "k + m must be <= 2^w - 1");
  if (m > kMaxM || k + m > kMaxBlocks)
    return fail(RS_EUNSUPPORTED, "device path limits: m <= 8 and k + m <= 64");
  rs_code* c = new (std::nothrow) rs_code();
  if (!c) return fail(RS_ENOMEM, "host allocation failed");
  c->k = k;
  c->m = m;
  c->w = w;
  c->real = (Realization)realization;
  if (c->real == Realization::Vandermonde) {
    if (!vandermonde_parity_matrix(k, m, w, c->P)) {
      delete c;
      return fail(RS_EINVAL, "Vandermonde construction failed");
    }
  } else if (c->real == Realization::Cauchy) {
    cauchy_parity_matrix(k, m, w, c->P);
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    if (c->d_status) cudaFree(c->d_status);
    delete c;
    return cuda_fail(e, "rs_init");
  }
  *out = c;
  return ok();
}

void rs_destroy(rs_code* c) {
  if (!c) return;
  if (c->d_status) cudaFree(c->d_status);
  delete c;
}

rs_status rs_set_packet_bytes(rs_code* c, size_t packet_bytes) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (c->real != Realization::Cauchy) return fail(RS_EINVAL, "packet size applies to the Cauchy realization only");
  if (packet_bytes == 0 || packet_bytes % 16) return fail(RS_EINVAL, "packet_bytes must be a positive multiple of 16");
  c->packet_bytes = packet_bytes;
  return ok();
}

rs_status rs_set_read_mode(rs_code* c, int mode) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (mode != RS_READ_MIN && mode != RS_READ_ALL) return fail(RS_EINVAL, "unknown read mode");
  c->read_mode = mode;
  return ok();
}

rs_status rs_set_launch(rs_code* c, int consumer_warps, int depth, int ctas_per_sm) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (consumer_warps < 0 || consumer_warps > 16 || depth < 0 || depth > 64 || ctas_per_sm < 0 || ctas_per_sm > 4 ||
      (depth != 0 && depth < 2))
    return fail(RS_EINVAL, "launch shape out of range");
  if (consumer_warps) c->tune.consumer_warps = consumer_warps;
  if (depth) c->tune.depth = depth;
  if (ctas_per_sm) c->tune.ctas_per_sm = ctas_per_sm;
  return ok();
}

rs_status rs_encode(rs_code* c, const void* const* data_ptrs, void* const* parity_ptrs, size_t block_bytes,
                    void* stream) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (!data_ptrs || !parity_ptrs) return fail(RS_EINVAL, "pointer array is null");
  std::vector<const void*> all;
  for (int i = 0; i < c->k; ++i) all.push_back(data_ptrs[i]);
  for (int j = 0; j < c->m; ++j) all.push_back(parity_ptrs[j]);
  rs_status s = check_blocks(c, all, block_bytes);
  if (s != RS_OK) return s;
  if ((s = check_device(c)) != RS_OK) return s;
  if (block_bytes == 0) return ok();
  if (c->real != Realization::Poly) return fail(RS_EUNSUPPORTED, "realization not available in this build");

  JobParams* p = new (std::nothrow) JobParams();
  if (!p) return fail(RS_ENOMEM, "host allocation failed");
  uint32_t slice, depth;
  const int cap = poly_max_consumer_warps(c->w, c->m, kOpEncode);
  const int nc = std::max(1, std::min(c->tune.consumer_warps, cap));
  const uint32_t seg = (uint32_t)nc * segment_bytes(c->w);
  const uint32_t tiles = (uint32_t)((block_bytes + seg - 1) / seg);
  LaunchShape sh = make_shape(c, cap, tiles, slice, depth);
  p->status = c->d_status;
  p->n_stripes = 1;
  p->total_tiles = tiles;
  p->slice_bytes = slice;
  p->depth = depth;
  StripeDesc& d = p->inl_stripe;
  d.bytes = block_bytes;
  d.tile_begin = 0;
  d.ptr_off = 0;
  d.n_in = (uint16_t)c->k;
  d.n_out = (uint16_t)c->m;
  d.op = kOpEncode;
  d.m = (uint8_t)c->m;
  d.k = (uint8_t)c->k;
  d.layout = kLayoutSymbol;
  for (int i = 0; i < c->k; ++i) p->inl_ptrs[i] = (uint64_t)(uintptr_t)data_ptrs[c->k - 1 - i];
  for (int j = 0; j < c->m; ++j) p->inl_ptrs[c->k + j] = (uint64_t)(uintptr_t)parity_ptrs[j];
  cudaError_t e = launch_poly(c->w, c->m, kOpEncode, *p, sh, (cudaStream_t)stream);
  delete p;
  if (e != cudaSuccess) return cuda_fail(e, "encode launch");
  return ok();
}

rs_status rs_decode(rs_code* c, const int* erasures, int n_erasures, void* const* block_ptrs, size_t block_bytes,
                    void* stream) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (n_erasures < 0) return fail(RS_EINVAL, "negative erasure count");
  if (n_erasures > c->m) return fail(RS_ETOOMANY_ERASURES, "more erasures than parity blocks");
  if (n_erasures > 0 && !erasures) return fail(RS_EINVAL, "erasure list is null");
  if (!block_ptrs) return fail(RS_EINVAL, "pointer array is null");
  const int n = c->k + c->m;
  std::vector<const void*> all;
  for (int b = 0; b < n; ++b) all.push_back(block_ptrs[b]);
  rs_status s = check_blocks(c, all, block_bytes);
  if (s != RS_OK) return s;
  if ((s = check_device(c)) != RS_OK) return s;
  const DecodePlan* pl = nullptr;
  if ((s = get_plan(c, erasures, n_erasures, &pl)) != RS_OK) return s;
  if (n_erasures == 0 || block_bytes == 0) return ok();
  if (c->real != Realization::Poly) return fail(RS_EUNSUPPORTED, "realization not available in this build");

  JobParams* p = new (std::nothrow) JobParams();
  if (!p) return fail(RS_ENOMEM, "host allocation failed");
  uint32_t slice, depth;
  const int cap = poly_max_consumer_warps(c->w, pl->M, kOpDecode);
  const int nc = std::max(1, std::min(c->tune.consumer_warps, cap));
  const uint32_t seg = (uint32_t)nc * segment_bytes(c->w);
  const uint32_t tiles = (uint32_t)((block_bytes + seg - 1) / seg);
  LaunchShape sh = make_shape(c, cap, tiles, slice, depth);
  p->status = c->d_status;
  p->n_stripes = 1;
  p->total_tiles = tiles;
  p->slice_bytes = slice;
  p->depth = depth;
  StripeDesc& d = p->inl_stripe;
  d.bytes = block_bytes;
  d.read_mask = pl->read_mask;
  d.n_in = (uint16_t)pl->in_blocks.size();
  d.n_out = (uint16_t)pl->e;
  d.op = kOpDecode;
  d.m = (uint8_t)pl->M;
  d.n_pos = (uint8_t)pl->n_pos;
  d.e = (uint8_t)pl->e;
  d.k = (uint8_t)c->k;
  d.layout = kLayoutSymbol;
  d.coef_off = 0;
  size_t q = 0;
  for (int b : pl->in_blocks) p->inl_ptrs[q++] = (uint64_t)(uintptr_t)block_ptrs[b];
  for (int b : pl->out_blocks) p->inl_ptrs[q++] = (uint64_t)(uintptr_t)block_ptrs[b];
  fill_masks(p->inl_coef, *pl, c->w);
  cudaError_t e = launch_poly(c->w, pl->M, kOpDecode, *p, sh, (cudaStream_t)stream);
  delete p;
  if (e != cudaSuccess) return cuda_fail(e, "decode launch");
  return ok();
}

rs_status rs_poll_status(rs_code* c, int* device_status) {
  if (!c) return fail(RS_EINVAL, "code is null");
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "rs_poll_status");
  if (v) {
    e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "rs_poll_status");
  }
  if (device_status) *device_status = v;
  return v ? fail(RS_ETIMEOUT, "device-side wait timed out (status " + std::to_string(v) + ")") : ok();
}

}  // extern "C"
