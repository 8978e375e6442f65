// C ABI of the library (declared in include/rs_gb300.h): argument checks,
// per-code generator construction, decode-plan cache, single-stripe calls
// and batches of stripe operations.
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
#include "registry.hpp"
#include "tile_geom.hpp"
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

constexpr int kMaxGroups = 8;                        // kernels per batch launch
// Batches whose polynomial ops move at most this many bytes use the mixed
// polynomial kernel (at ~5 TB/s about 50 us of work: a few launches' worth).
constexpr uint64_t kMixedMaxBytes = 256ull << 20;
constexpr int kKindOf[6] = {0, kKindVandermonde, kKindCauchy, kKindPolyMatrix, kKindPolyBitMatrix, kKindGoodCauchy};

bool packet_layout(Realization r) {
  return r == Realization::Cauchy || r == Realization::PolyBitMatrix || r == Realization::GoodCauchy;
}

bool has_fixed_kernels(int w, int k, int m, int kind) {
  KernelKey key;
  key.family = kFamMatFixed;
  key.w = w;
  key.m = m;
  key.op = kOpMatEncode;
  key.layout = kind_layout(kind);
  key.kind = kind;
  key.k = k;
  return find_kernel(key) != nullptr;
}

}  // namespace

namespace rsgb {
void set_last_error(const std::string& msg) { g_last_error = msg; }
void clear_last_error() { g_last_error.clear(); }
}  // namespace rsgb

struct rs_code {
  int k = 0, m = 0, w = 0;
  Realization real = Realization::Poly;
  size_t packet_bytes = 2048;
  int read_mode = RS_READ_MIN;
  TuneCfg tune;
  std::vector<uint32_t> P;       // parity rows of the generator (matrix realizations)
  uint32_t* d_pmask = nullptr;   // column masks of P on the device (runtime-P kernels)
  uint32_t* d_update = nullptr;  // per data index i: columns [P[:, i] | I_m] as bits (rs_update)
  bool fixed = false;            // compile-time-P kernels exist for (w, k, m)
  int device = 0;
  int num_sms = 0;
  int* d_status = nullptr;
  unsigned long long wait_limit_ns = 0;  // 0: kernel default
  uint32_t inject_next = 0;              // test hook for the next launch
  std::mutex mu;
  std::map<std::vector<int>, DecodePlan> plans;  // key: read mode, erasure list
};

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

rs_status check_device(int device) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != device)
    return fail(RS_EINVAL, "object was created on device " + std::to_string(device) + " but device " +
                               std::to_string(dev) + " is current");
  return RS_OK;
}

// Blocks of one operation must be pairwise disjoint.
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
  if (bytes == 0) return RS_OK;  // nothing is read or written: any pointers do
  for (size_t i = 0; i < ptrs.size(); ++i) {
    if (!ptrs[i]) return fail(RS_EINVAL, "null block pointer");
    if (!aligned16(ptrs[i])) return fail(RS_EINVAL, "block pointers must be 16-byte aligned");
  }
  if (c->w == 16 && (bytes & 1u)) return fail(RS_EINVAL, "block_bytes must be even for w = 16");
  if (packet_layout(c->real) && bytes % ((size_t)c->w * c->packet_bytes))
    return fail(RS_EINVAL, "block_bytes must be a multiple of w * packet_bytes for the bit-matrix realizations");
  if (bytes > ((size_t)1 << 40)) return fail(RS_EINVAL, "block_bytes too large");
  if (!disjoint(ptrs, bytes)) return fail(RS_EINVAL, "blocks of one operation must not overlap");
  return RS_OK;
}

rs_status get_plan(rs_code* c, const int* er, int e, DecodePlan& out) {
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
  out = it->second;
  return RS_OK;
}

// One stripe operation, ready for a kernel: descriptor (tile_begin,
// ptr_off, coef_off filled in by the launcher), pointers and masks.
struct PreparedOp {
  KernelKey key;
  const KernelEntry* entry = nullptr;
  StripeDesc d{};
  std::vector<uint64_t> ptrs;
  std::vector<uint32_t> coef;
  bool noop = false;
};

// Two-column-group kernels (KernelKey::wide) cover twice the columns per
// tile; below these block sizes the coarser tiles leave warps idle on the
// ragged last tile of every block and the one-group kernel measured faster.
constexpr size_t kWideSymbolMinBytes = 256u << 10;
constexpr size_t kWidePacketMinBytes = 8u << 10;

// groups: 0 = the two-group kernel from the thresholds above, 1 = the
// one-group kernel, 2 = the two-group kernel whenever one is compiled.
rs_status select_kernel(const rs_code* c, int op, int M, size_t B, PreparedOp& po, int groups) {
  KernelKey key;
  key.w = c->w;
  key.m = M;
  if (c->real == Realization::Poly) {
    key.family = kFamPoly;
    key.op = op;  // kOpEncode / kOpDecode
  } else {
    key.op = op == kOpEncode ? kOpMatEncode : kOpMatDecode;
    key.layout = packet_layout(c->real) ? kLayoutPacket : kLayoutSymbol;
    if (c->fixed) {
      key.family = kFamMatFixed;
      key.kind = kKindOf[(int)c->real];
      key.k = c->k;
    } else {
      key.family = kFamMatRuntime;
    }
  }
  po.entry = nullptr;
  const size_t wide_min = key.layout == kLayoutPacket ? kWidePacketMinBytes : kWideSymbolMinBytes;
  if (groups == 2 || (groups == 0 && B >= wide_min)) {
    key.wide = 1;
    po.entry = find_kernel(key);
    // a packet kernel's tiles are whole warps of units (G 32-bit words of
    // each packet row), so its packets must hold a multiple of 32 units
    if (po.entry && key.layout == kLayoutPacket && c->packet_bytes % (size_t)(128 * po.entry->groups))
      po.entry = nullptr;
    if (!po.entry) key.wide = 0;
  }
  if (!po.entry) po.entry = find_kernel(key);
  po.key = key;
  if (!po.entry) return fail(RS_EUNSUPPORTED, "no kernel compiled for this code");
  return RS_OK;
}

void fill_common(const rs_code* c, size_t B, StripeDesc& d) {
  d.bytes = B;
  d.k = (uint8_t)c->k;
  d.layout = packet_layout(c->real) ? kLayoutPacket : kLayoutSymbol;
  d.packet_bytes = packet_layout(c->real) ? (uint32_t)c->packet_bytes : 0u;
  d.pmask = (uint64_t)(uintptr_t)c->d_pmask;
}

rs_status prepare_encode(rs_code* c, const void* const* data, void* const* parity, size_t B, PreparedOp& po,
                         int groups) {
  if (!data || !parity) return fail(RS_EINVAL, "pointer array is null");
  std::vector<const void*> all;
  for (int i = 0; i < c->k; ++i) all.push_back(data[i]);
  for (int j = 0; j < c->m; ++j) all.push_back(parity[j]);
  rs_status s = check_blocks(c, all, B);
  if (s != RS_OK) return s;
  if ((s = select_kernel(c, kOpEncode, c->m, B, po, groups)) != RS_OK) return s;
  po.noop = B == 0;
  StripeDesc& d = po.d;
  fill_common(c, B, d);
  d.n_in = (uint16_t)c->k;
  d.n_out = (uint16_t)c->m;
  d.op = (uint8_t)po.key.op;
  d.m = (uint8_t)c->m;
  po.ptrs.clear();
  if (c->real == Realization::Poly) {
    // LFSR consumption order: d_{k-1} first (highest degree, §3.2 Eq. 2)
    for (int i = c->k - 1; i >= 0; --i) po.ptrs.push_back((uint64_t)(uintptr_t)data[i]);
  } else {
    for (int i = 0; i < c->k; ++i) po.ptrs.push_back((uint64_t)(uintptr_t)data[i]);
  }
  for (int j = 0; j < c->m; ++j) po.ptrs.push_back((uint64_t)(uintptr_t)parity[j]);
  po.coef.clear();
  return RS_OK;
}

// Delta update (§3.2's update remark: the encode of the data diff-blocks is
// the parity diff): data block `index` changed by delta, so parity block j
// gains P[j][index] * delta.  Run as the runtime-matrix encode of the m + 1
// inputs (delta, p_0 .. p_(m-1)) by U = [P[:, index] | I_m], the outputs
// written over p_0 .. p_(m-1): every tile reads its slice of a block before
// it writes the same slice, and no other tile touches those bytes.
rs_status prepare_update(rs_code* c, int index, const void* delta, void* const* parity, size_t B, PreparedOp& po) {
  if (index < 0 || index >= c->k) return fail(RS_EINVAL, "data index out of range");
  if (!parity) return fail(RS_EINVAL, "pointer array is null");
  std::vector<const void*> all{delta};
  for (int j = 0; j < c->m; ++j) all.push_back(parity[j]);
  rs_status s = check_blocks(c, all, B);
  if (s != RS_OK) return s;
  KernelKey key;
  key.family = kFamMatRuntime;
  key.w = c->w;
  key.m = c->m;
  key.op = kOpMatEncode;
  key.layout = packet_layout(c->real) ? kLayoutPacket : kLayoutSymbol;
  po.key = key;
  po.entry = find_kernel(key);
  if (!po.entry) return fail(RS_EUNSUPPORTED, "no kernel compiled for this code");
  po.noop = B == 0;
  StripeDesc& d = po.d;
  fill_common(c, B, d);
  d.k = (uint8_t)(c->m + 1);
  d.pmask = (uint64_t)(uintptr_t)(c->d_update + (size_t)index * (c->m + 1) * column_words(c->m, c->w));
  d.n_in = (uint16_t)(c->m + 1);
  d.n_out = (uint16_t)c->m;
  d.op = (uint8_t)kOpMatEncode;
  d.m = (uint8_t)c->m;
  po.ptrs.clear();
  po.ptrs.push_back((uint64_t)(uintptr_t)delta);
  for (int j = 0; j < c->m; ++j) po.ptrs.push_back((uint64_t)(uintptr_t)parity[j]);
  for (int j = 0; j < c->m; ++j) po.ptrs.push_back((uint64_t)(uintptr_t)parity[j]);
  po.coef.clear();
  return RS_OK;
}

rs_status prepare_decode(rs_code* c, const int* er, int e, void* const* blocks, size_t B, PreparedOp& po,
                         int groups) {
  if (e < 0) return fail(RS_EINVAL, "negative erasure count");
  if (e > c->m) return fail(RS_ETOOMANY_ERASURES, "more erasures than parity blocks");
  if (e > 0 && !er) return fail(RS_EINVAL, "erasure list is null");
  if (!blocks) return fail(RS_EINVAL, "pointer array is null");
  const int n = c->k + c->m;
  std::vector<const void*> all;
  for (int b = 0; b < n; ++b) all.push_back(blocks[b]);
  rs_status s = check_blocks(c, all, B);
  if (s != RS_OK) return s;
  DecodePlan pl;
  if ((s = get_plan(c, er, e, pl)) != RS_OK) return s;
  po.noop = e == 0 || B == 0;
  if (e == 0) return RS_OK;
  if ((s = select_kernel(c, kOpDecode, pl.M, B, po, groups)) != RS_OK) return s;
  StripeDesc& d = po.d;
  fill_common(c, B, d);
  d.read_mask = pl.read_mask;
  d.n_in = (uint16_t)pl.in_blocks.size();
  d.n_out = (uint16_t)pl.e;
  d.op = (uint8_t)po.key.op;
  d.m = (uint8_t)pl.M;
  d.n_pos = (uint8_t)pl.n_pos;
  d.e = (uint8_t)pl.e;
  po.ptrs.clear();
  for (int b : pl.in_blocks) po.ptrs.push_back((uint64_t)(uintptr_t)blocks[b]);
  for (int b : pl.out_blocks) po.ptrs.push_back((uint64_t)(uintptr_t)blocks[b]);
  po.coef = pack_decode_selectors(pl, c->w);
  while (po.coef.size() % 4) po.coef.push_back(0u);  // keep every op's words 16-byte aligned
  return RS_OK;
}

// Consumer warps for a launch: the tuned value capped by the kernel (a
// multiple of 4 for kernels with a producer warpgroup).
int pick_warps(const TuneCfg& t, const KernelEntry* e) {
  int nc = std::max(1, std::min(t.consumer_warps, e->max_warps));
  if (e->producer_warps == 4) nc = std::max(4, nc / 4 * 4);
  return nc;
}

// A launch's geometry.  slice = one block's bytes of a tile; slot = the
// ring's slot stride.  Packet tiles copy the whole super-packets they touch
// (one bulk copy per block instead of one per packet row of a partial
// super-packet) when those take at most 3 times the tile's own bytes and a
// ring of two such slots fits shared memory; `whole` reports that choice.
// The extra bytes are the neighbouring tiles' parts of the same
// super-packets, which the same CTA reads next (L2 hits); many small bulk
// copies cost more: GF(2^16) RS(12,4) good Cauchy encode 3677 GB/s with the
// per-row copies, 5676 with whole super-packets at up to 2.1 times the
// bytes.
LaunchShape make_shape(const TuneCfg& t, int nc, int pw, int w, int groups, int num_sms, int layout,
                       const std::vector<uint32_t>& packets, uint32_t& slice, uint32_t& slot, uint32_t& depth,
                       uint32_t& whole) {
  slice = (uint32_t)(nc * groups) * segment_bytes(w);
  slot = slice;
  whole = 0;
  if (layout == kLayoutPacket && !packets.empty()) {
    uint32_t need = slice;
    bool fits = true;
    for (uint32_t pb : packets) {
      const uint32_t wb = packet_whole_bytes(slice, w, groups, pb);
      fits = fits && wb <= 3ull * slice && ring_smem_bytes(2, wb) <= kMaxDynamicSmem;
      need = std::max(need, wb);
    }
    if (fits) {
      whole = 1;
      slot = need;
    }
  }
  depth = (uint32_t)std::max(2, t.depth);
  const size_t budget = kMaxDynamicSmem / (size_t)std::max(1, t.ctas_per_sm);
  while (depth > 2 && ring_smem_bytes(depth, slot) > budget) --depth;
  LaunchShape sh;
  sh.threads = (nc + pw) * 32;
  sh.smem = ring_smem_bytes(depth, slot);
  sh.grid = std::max(1, num_sms * std::max(1, t.ctas_per_sm));
  return sh;
}

uint32_t tiles_of(const StripeDesc& d, uint32_t slice) {
  return (uint32_t)((d.bytes + slice - 1) / slice);
}

rs_status launch_single(rs_code* c, PreparedOp& po, void* stream) {
  if (po.noop) return ok();
  rs_status s = check_device(c->device);
  if (s != RS_OK) return s;
  JobParams* p = new (std::nothrow) JobParams();
  if (!p) return fail(RS_ENOMEM, "host allocation failed");
  const int nc = pick_warps(c->tune, po.entry);
  uint32_t slice, slot, depth, whole;
  LaunchShape sh = make_shape(c->tune, nc, po.entry->producer_warps, c->w, po.entry->groups, c->num_sms, po.key.layout, {po.d.packet_bytes},
                              slice, slot, depth, whole);
  p->status = c->d_status;
  p->n_stripes = 1;
  p->slice_bytes = slice;
  p->slot_bytes = slot;
  p->packet_whole = whole;
  p->depth = depth;
  p->wait_limit_ns = c->wait_limit_ns;
  p->inject = c->inject_next;
  c->inject_next = 0;
  p->inl_stripe = po.d;
  p->inl_stripe.tile_begin = 0;
  p->inl_stripe.ptr_off = 0;
  p->inl_stripe.coef_off = 0;
  p->total_tiles = tiles_of(po.d, slice);
  sh.grid = (int)std::min<uint32_t>((uint32_t)sh.grid, p->total_tiles);
  std::copy(po.ptrs.begin(), po.ptrs.end(), p->inl_ptrs);
  std::copy(po.coef.begin(), po.coef.end(), p->inl_coef);
  cudaError_t e = po.entry->launch(*p, sh, (cudaStream_t)stream);
  delete p;
  if (e != cudaSuccess) return cuda_fail(e, po.entry->name);
  return ok();
}

}  // namespace

// ------------------------------------------------------------------ batches
struct rs_batch {
  int max_ops = 0;
  int device = 0;
  int num_sms = 0;
  TuneCfg tune;
  StripeDesc* d_stripes = nullptr;  // kMaxGroups regions of max_ops
  uint64_t* d_ptrs = nullptr;       // max_ops * kMaxPtrs
  uint32_t* d_coef = nullptr;       // max_ops * kMaxCoefWords
  uint32_t* d_counts = nullptr;     // kMaxGroups * 2
  int* d_status = nullptr;
  uint8_t* h_stage = nullptr;       // pinned upload staging
  size_t stage_bytes = 0;
  cudaEvent_t uploaded = nullptr;
  bool upload_pending = false;
  // kernel groups after the first run on side streams forked from and
  // joined back into the launch stream, so that a group's kernel fills the
  // SMs that another group's tail leaves idle
  cudaStream_t side[kMaxGroups - 1] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kMaxGroups - 1] = {};
  struct Group {
    const KernelEntry* entry;
    int layout;
    int nc;
    uint32_t slice, slot, depth, whole;
    uint32_t n_stripes, tiles;
    LaunchShape sh;
  };
  std::vector<Group> groups;
};

namespace {

size_t stage_layout(int max_ops, size_t* off_ptrs, size_t* off_coef, size_t* off_counts) {
  size_t o = sizeof(StripeDesc) * (size_t)kMaxGroups * max_ops;
  *off_ptrs = o;
  o += sizeof(uint64_t) * (size_t)max_ops * kMaxPtrs;
  *off_coef = o;
  o += sizeof(uint32_t) * (size_t)max_ops * kMaxCoefWords;
  *off_counts = o;
  o += sizeof(uint32_t) * kMaxGroups * 2;
  return o;
}

void batch_free(rs_batch* b) {
  for (int i = 0; i < kMaxGroups - 1; ++i) {
    if (b->side[i]) cudaStreamDestroy(b->side[i]);
    if (b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_stripes) cudaFree(b->d_stripes);
  if (b->d_ptrs) cudaFree(b->d_ptrs);
  if (b->d_coef) cudaFree(b->d_coef);
  if (b->d_counts) cudaFree(b->d_counts);
  if (b->d_status) cudaFree(b->d_status);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->uploaded) cudaEventDestroy(b->uploaded);
}

// Kernel used for an op inside a batch: a mixed polynomial kernel replaces
// per-M kernels when the batch holds several M it covers.
const KernelEntry* mixed_for(const KernelKey& k) {
  if (k.family != kFamPoly) return nullptr;
  for (int i = 0; i < kKernelRegistrySize; ++i) {
    const KernelEntry& e = kKernelRegistryPtr[i];
    if (e.key.family == kFamPolyMixed && e.key.w == k.w && ((e.key.mset >> k.m) & 1u)) return &e;
  }
  return nullptr;
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
  if (realization < RS_POLY || realization > RS_GOOD_CAUCHY) return fail(RS_EINVAL, "unknown realization");
  if ((long)k + m > (1L << w) - 1) return fail(RS_EINVAL, "k + m must be <= 2^w - 1");
  if (m > kMaxM || k + m > kMaxBlocks || (w == 16 && m > 4))
    return fail(RS_EUNSUPPORTED, "device path limits: m <= 8 (m <= 4 for w = 16) and k + m <= 64");
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
  } else if (c->real == Realization::GoodCauchy) {
    good_cauchy_parity_matrix(k, m, w, c->P);
  } else {
    // polynomial code (any of its three realizations): column i of P is
    // x^(m+i) mod g(x), the parity of the unit data vector e_i
    poly_parity_matrix(k, m, w, c->P);
  }
  c->fixed = c->real != Realization::Poly && has_fixed_kernels(w, k, m, kKindOf[(int)c->real]);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e == cudaSuccess && c->real != Realization::Poly) {
    // P's columns as packed bits for the runtime-P kernels
    const std::vector<uint32_t> masks = pack_columns(c->P, k, m, w);
    e = cudaMalloc(&c->d_pmask, masks.size() * sizeof(uint32_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_pmask, masks.data(), masks.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    // update matrices U_i = [P[:, i] | I_m] (m x (m + 1)), one after another
    std::vector<uint32_t> all;
    std::vector<uint32_t> U((size_t)m * (m + 1));
    for (int i = 0; i < k; ++i) {
      for (int j = 0; j < m; ++j) {
        U[(size_t)j * (m + 1)] = c->P[(size_t)j * k + i];
        for (int l = 0; l < m; ++l) U[(size_t)j * (m + 1) + 1 + l] = j == l ? 1u : 0u;
      }
      const std::vector<uint32_t> cols = pack_columns(U, m + 1, m, w);
      all.insert(all.end(), cols.begin(), cols.end());
    }
    e = cudaMalloc(&c->d_update, all.size() * sizeof(uint32_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_update, all.data(), all.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_pmask) cudaFree(c->d_pmask);
    if (c->d_update) cudaFree(c->d_update);
    delete c;
    return cuda_fail(e, "rs_init");
  }
  *out = c;
  return ok();
}

void rs_destroy(rs_code* c) {
  if (!c) return;
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_pmask) cudaFree(c->d_pmask);
  if (c->d_update) cudaFree(c->d_update);
  delete c;
}

rs_status rs_set_packet_bytes(rs_code* c, size_t packet_bytes) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (!packet_layout(c->real)) return fail(RS_EINVAL, "packet size applies to the bit-matrix realizations only");
  if (packet_bytes == 0 || packet_bytes % 128 || packet_bytes > (1u << 20))
    return fail(RS_EINVAL, "packet_bytes must be a positive multiple of 128 (at most 1 MiB)");
  c->packet_bytes = packet_bytes;
  return ok();
}

rs_status rs_set_read_mode(rs_code* c, int mode) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (mode != RS_READ_MIN && mode != RS_READ_ALL) return fail(RS_EINVAL, "unknown read mode");
  c->read_mode = mode;
  return ok();
}

static rs_status set_tune(TuneCfg& t, int consumer_warps, int depth, int ctas_per_sm) {
  if (consumer_warps < 0 || consumer_warps > 16 || depth < 0 || depth > 64 || ctas_per_sm < 0 || ctas_per_sm > 4 ||
      (depth != 0 && depth < 2))
    return fail(RS_EINVAL, "launch shape out of range");
  if (consumer_warps) t.consumer_warps = consumer_warps;
  if (depth) t.depth = depth;
  if (ctas_per_sm) t.ctas_per_sm = ctas_per_sm;
  return ok();
}

rs_status rs_set_launch(rs_code* c, int consumer_warps, int depth, int ctas_per_sm) {
  if (!c) return fail(RS_EINVAL, "code is null");
  return set_tune(c->tune, consumer_warps, depth, ctas_per_sm);
}

rs_status rs_set_groups(rs_code* c, int groups) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (groups < 0 || groups > 2) return fail(RS_EINVAL, "groups must be 0, 1 or 2");
  c->tune.groups = groups;
  return ok();
}

rs_status rs_encode(rs_code* c, const void* const* data_ptrs, void* const* parity_ptrs, size_t block_bytes,
                    void* stream) {
  if (!c) return fail(RS_EINVAL, "code is null");
  PreparedOp po;
  rs_status s = prepare_encode(c, data_ptrs, parity_ptrs, block_bytes, po, c->tune.groups);
  if (s != RS_OK) return s;
  return launch_single(c, po, stream);
}

rs_status rs_decode(rs_code* c, const int* erasures, int n_erasures, void* const* block_ptrs, size_t block_bytes,
                    void* stream) {
  if (!c) return fail(RS_EINVAL, "code is null");
  PreparedOp po;
  rs_status s = prepare_decode(c, erasures, n_erasures, block_ptrs, block_bytes, po, c->tune.groups);
  if (s != RS_OK) return s;
  return launch_single(c, po, stream);
}

rs_status rs_update(rs_code* c, int index, const void* delta, void* const* parity_ptrs, size_t block_bytes,
                    void* stream) {
  if (!c) return fail(RS_EINVAL, "code is null");
  PreparedOp po;
  rs_status s = prepare_update(c, index, delta, parity_ptrs, block_bytes, po);
  if (s != RS_OK) return s;
  return launch_single(c, po, stream);
}

rs_status rs_set_wait_limit(rs_code* c, unsigned long long nanoseconds) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (nanoseconds > 60ull * 1000000000ull) return fail(RS_EINVAL, "wait limit above 60 s");
  c->wait_limit_ns = nanoseconds;
  return ok();
}

rs_status rs_inject_fault(rs_code* c, int fault) {
  if (!c) return fail(RS_EINVAL, "code is null");
  if (fault != 0 && fault != (int)kInjectProducerStall) return fail(RS_EINVAL, "unknown fault");
  c->inject_next = (uint32_t)fault;
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

// ------------------------------------------------------------ batch API
rs_status rs_batch_create(int max_ops, rs_batch** out) {
  if (!out) return fail(RS_EINVAL, "out is null");
  *out = nullptr;
  if (max_ops < 1 || max_ops > (1 << 20)) return fail(RS_EINVAL, "max_ops must be in [1, 2^20]");
  rs_batch* b = new (std::nothrow) rs_batch();
  if (!b) return fail(RS_ENOMEM, "host allocation failed");
  b->max_ops = max_ops;
  size_t op, oc, ocn;
  b->stage_bytes = stage_layout(max_ops, &op, &oc, &ocn);
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_stripes, sizeof(StripeDesc) * (size_t)kMaxGroups * max_ops);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ptrs, sizeof(uint64_t) * (size_t)max_ops * kMaxPtrs);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_coef, sizeof(uint32_t) * (size_t)max_ops * kMaxCoefWords);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counts, sizeof(uint32_t) * kMaxGroups * 2);
  if (e == cudaSuccess) e = cudaMemset(b->d_counts, 0, sizeof(uint32_t) * kMaxGroups * 2);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_stage, b->stage_bytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < kMaxGroups - 1 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? fail(RS_ENOMEM, "batch allocation failed") : cuda_fail(e, "rs_batch_create");
  }
  *out = b;
  return ok();
}

void rs_batch_destroy(rs_batch* b) {
  if (!b) return;
  batch_free(b);
  delete b;
}

rs_status rs_batch_set_launch(rs_batch* b, int consumer_warps, int depth, int ctas_per_sm) {
  if (!b) return fail(RS_EINVAL, "batch is null");
  return set_tune(b->tune, consumer_warps, depth, ctas_per_sm);
}

rs_status rs_batch_set_groups(rs_batch* b, int groups) {
  if (!b) return fail(RS_EINVAL, "batch is null");
  if (groups < 0 || groups > 2) return fail(RS_EINVAL, "groups must be 0, 1 or 2");
  b->tune.groups = groups;
  return ok();
}

rs_status rs_batch_set(rs_batch* b, const rs_op* ops, int n_ops, void* stream) {
  if (!b) return fail(RS_EINVAL, "batch is null");
  if (n_ops < 0 || n_ops > b->max_ops) return fail(RS_EINVAL, "n_ops out of range");
  if (n_ops > 0 && !ops) return fail(RS_EINVAL, "ops is null");
  rs_status s = check_device(b->device);
  if (s != RS_OK) return s;
  // prepare every op
  std::vector<PreparedOp> prep(n_ops);
  for (int i = 0; i < n_ops; ++i) {
    const rs_op& o = ops[i];
    if (!o.code) return fail(RS_EINVAL, "op " + std::to_string(i) + ": code is null");
    if (o.code->device != b->device) return fail(RS_EINVAL, "op " + std::to_string(i) + ": code on another device");
    if (o.op == RS_OP_ENCODE)
      s = prepare_encode(o.code, (const void* const*)o.blocks, (void* const*)(o.blocks + o.code->k), o.block_bytes,
                         prep[i], b->tune.groups);
    else if (o.op == RS_OP_DECODE)
      s = prepare_decode(o.code, o.erasures, o.n_erasures, o.blocks, o.block_bytes, prep[i], b->tune.groups);
    else
      s = fail(RS_EINVAL, "unknown op kind");
    if (s != RS_OK) return fail(s, "op " + std::to_string(i) + ": " + g_last_error);
  }
  // group by kernel (mixed polynomial kernels merge several M)
  std::vector<const KernelEntry*> group_entry;
  std::vector<std::vector<int>> members;
  // A mixed polynomial kernel (one launch for several M and both ops)
  // replaces the per-M kernels only for small batches, where the launches
  // it saves matter; large ones keep the specialised kernels (more warps,
  // two column groups for the decodes).
  std::map<const KernelEntry*, uint64_t> primary_bytes;
  for (auto& po : prep)
    if (!po.noop) primary_bytes[po.entry] += (uint64_t)(po.d.n_in + po.d.n_out) * po.d.bytes;
  std::map<const KernelEntry*, int> mixed_users;
  std::map<const KernelEntry*, uint64_t> mixed_bytes;
  for (auto& kv : primary_bytes) {
    const KernelEntry* mx = mixed_for(kv.first->key);
    if (!mx) continue;
    mixed_users[mx]++;
    mixed_bytes[mx] += kv.second;
  }
  for (int i = 0; i < n_ops; ++i) {
    if (prep[i].noop) continue;
    const KernelEntry* e = prep[i].entry;
    const KernelEntry* mx = mixed_for(e->key);
    if (mx && mixed_users[mx] >= 2 && mixed_bytes[mx] <= kMixedMaxBytes) e = mx;
    int g = -1;
    for (size_t j = 0; j < group_entry.size(); ++j)
      if (group_entry[j] == e) g = (int)j;
    if (g < 0) {
      if ((int)group_entry.size() == kMaxGroups) return fail(RS_EUNSUPPORTED, "more than 8 kernel groups in one batch");
      group_entry.push_back(e);
      members.emplace_back();
      g = (int)group_entry.size() - 1;
    }
    members[g].push_back(i);
  }
  // wait until the previous upload has left the staging buffer
  if (b->upload_pending) {
    cudaError_t e = cudaEventSynchronize(b->uploaded);
    if (e != cudaSuccess) return cuda_fail(e, "rs_batch_set");
    b->upload_pending = false;
  }
  size_t off_ptrs, off_coef, off_counts;
  stage_layout(b->max_ops, &off_ptrs, &off_coef, &off_counts);
  StripeDesc* hs = reinterpret_cast<StripeDesc*>(b->h_stage);
  uint64_t* hp = reinterpret_cast<uint64_t*>(b->h_stage + off_ptrs);
  uint32_t* hc = reinterpret_cast<uint32_t*>(b->h_stage + off_coef);
  uint32_t* hn = reinterpret_cast<uint32_t*>(b->h_stage + off_counts);
  memset(hn, 0, sizeof(uint32_t) * kMaxGroups * 2);
  size_t np = 0, ncw = 0;
  std::vector<rs_batch::Group> groups;
  for (size_t g = 0; g < group_entry.size(); ++g) {
    rs_batch::Group gr{};
    gr.entry = group_entry[g];
    const int layout = prep[members[g][0]].key.layout;
    gr.layout = layout;
    gr.nc = pick_warps(b->tune, gr.entry);
    const int w = gr.entry->key.w;
    std::vector<uint32_t> packets;
    if (layout == kLayoutPacket)
      for (int i : members[g]) packets.push_back(prep[i].d.packet_bytes);
    gr.sh = make_shape(b->tune, gr.nc, gr.entry->producer_warps, w, gr.entry->groups, b->num_sms, layout, packets, gr.slice, gr.slot, gr.depth,
                       gr.whole);
    uint64_t tiles = 0;  // tile numbers are 32-bit in the kernel
    StripeDesc* region = hs + g * (size_t)b->max_ops;
    for (size_t q = 0; q < members[g].size(); ++q) {
      PreparedOp& po = prep[members[g][q]];
      StripeDesc d = po.d;
      d.tile_begin = (uint32_t)tiles;
      d.ptr_off = (uint32_t)np;
      d.coef_off = (uint32_t)ncw;
      tiles += tiles_of(d, gr.slice);
      if (tiles > 0xFFFFFFFFull) return fail(RS_EINVAL, "too many tiles in one kernel group (more than 2^32)");
      std::copy(po.ptrs.begin(), po.ptrs.end(), hp + np);
      np += po.ptrs.size();
      std::copy(po.coef.begin(), po.coef.end(), hc + ncw);
      ncw += po.coef.size();
      region[q] = d;
    }
    gr.n_stripes = (uint32_t)members[g].size();
    gr.tiles = (uint32_t)tiles;
    hn[2 * g] = gr.n_stripes;
    hn[2 * g + 1] = gr.tiles;
    groups.push_back(gr);
  }
  // upload (stream-ordered)
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (size_t g = 0; g < groups.size() && e == cudaSuccess; ++g)
    e = cudaMemcpyAsync(b->d_stripes + g * (size_t)b->max_ops, hs + g * (size_t)b->max_ops,
                        sizeof(StripeDesc) * groups[g].n_stripes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && np) e = cudaMemcpyAsync(b->d_ptrs, hp, sizeof(uint64_t) * np, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && ncw)
    e = cudaMemcpyAsync(b->d_coef, hc, sizeof(uint32_t) * ncw, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_counts, hn, sizeof(uint32_t) * kMaxGroups * 2, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(b->uploaded, st);
  if (e != cudaSuccess) return cuda_fail(e, "rs_batch_set upload");
  b->upload_pending = true;
  b->groups = groups;
  return ok();
}

rs_status rs_batch_launch(rs_batch* b, void* stream) {
  if (!b) return fail(RS_EINVAL, "batch is null");
  rs_status s = check_device(b->device);
  if (s != RS_OK) return s;
  JobParams* p = new (std::nothrow) JobParams();
  if (!p) return fail(RS_ENOMEM, "host allocation failed");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ng = b->groups.size();
  if (ng > 1) {
    cudaError_t e = cudaEventRecord(b->fork, st);
    for (size_t g = 1; g < ng && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(b->side[g - 1], b->fork, 0);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "rs_batch_launch fork");
    }
  }
  for (size_t g = 0; g < ng; ++g) {
    const rs_batch::Group& gr = b->groups[g];
    p->stripes = b->d_stripes + g * (size_t)b->max_ops;
    p->ptrs = b->d_ptrs;
    p->coef = b->d_coef;
    p->counts = b->d_counts + 2 * g;
    p->status = b->d_status;
    p->n_stripes = gr.n_stripes;
    p->total_tiles = gr.tiles;
    p->slice_bytes = gr.slice;
    p->slot_bytes = gr.slot;
    p->packet_whole = gr.whole;
    p->depth = gr.depth;
    cudaStream_t gs = g == 0 ? st : b->side[g - 1];
    cudaError_t e = gr.entry->launch(*p, gr.sh, gs);
    if (e == cudaSuccess && g > 0) e = cudaEventRecord(b->join[g - 1], gs);
    if (e == cudaSuccess && g > 0) e = cudaStreamWaitEvent(st, b->join[g - 1], 0);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, gr.entry->name);
    }
  }
  delete p;
  return ok();
}

int rs_batch_kernel_count(const rs_batch* b) { return b ? (int)b->groups.size() : 0; }

rs_status rs_batch_poll_status(rs_batch* b, int* device_status) {
  if (!b) return fail(RS_EINVAL, "batch is null");
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "rs_batch_poll_status");
  if (v) {
    e = cudaMemset(b->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "rs_batch_poll_status");
  }
  if (device_status) *device_status = v;
  return v ? fail(RS_ETIMEOUT, "device-side wait timed out (status " + std::to_string(v) + ")") : ok();
}

}  // extern "C"
