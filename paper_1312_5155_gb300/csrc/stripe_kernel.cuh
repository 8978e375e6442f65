// Persistent, TMA-staged stripe kernel (sm_103a).
//
// CTA = NC consumer warps + 1 producer warp.  The producer's lane 0 walks the
// CTA's tiles (a contiguous run of the launch's global tile indices, so
// consecutive tiles almost always belong to the same stripe and the stripe's
// descriptor stays in registers) and, for every input block of the tile's
// stripe, issues 1-D bulk copies (cp.async.bulk) of the tile's slice of that
// block into the
// next slot of a shared-memory ring; the slot's full mbarrier counts the
// bytes.  Consumer warps walk the same tile sequence; every thread owns 32
// columns of the tile, reads them from the slot, runs the codec ("body") on
// bit-planes in registers and stores its output words straight to global
// memory.  Slots go back to the producer through the empty mbarriers (every
// consumer thread arrives once per slot use).
//
// Layouts
//   symbol: columns are bytes (w = 8) or little-endian 16-bit words
//     (w = 16).  Warp segment = 32 lanes x 32 symbols; lane l owns the
//     16-byte chunks at l*16 + c*512 (c < W/4) of its segment, so every
//     warp-wide load/store covers 512 contiguous bytes.  Slice of one block
//     per tile = NC segments, one bulk copy.
//   packet (§2.3 bit-matrix layout): a block is super-packets of W packets of
//     P bytes; packet c holds bit c of the super-packet's 8P symbols.  A
//     unit is G adjacent 32-bit words at the same offset of the W packets of
//     one super-packet (already the W bit-planes of 32G symbols); a block is
//     a sequence of units, super-packet after super-packet (U = P / 4G per
//     super-packet).  A tile covers NC*32 consecutive units, lane l of warp v
//     owning unit v*32 + l: a leading partial super-packet (W bulk copies
//     per block, one per packet row), whole super-packets (one bulk copy:
//     they are contiguous) and a trailing partial one (W copies).  The slot
//     holds the three parts one after the other, each row-major.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "codec_matrix.hpp"
#include "codec_poly.hpp"
#include "job.hpp"
#include "launch.hpp"
#include "pipeline.cuh"
#include "tile_geom.hpp"

namespace rsgb {

struct Ring {
  uint64_t* full;
  uint64_t* empty;
  uint8_t* slots;
  uint32_t depth;
  uint32_t slice;    // bytes of one block per tile (symbol layout)
  uint32_t stride;   // bytes between slots (>= slice)
  uint32_t s = 0;    // next slot
  uint32_t par = 0;  // parity of the next slot's current round
  __device__ __forceinline__ void advance() {
    if (++s == depth) {
      s = 0;
      par ^= 1u;
    }
  }
};

__device__ __forceinline__ uint32_t find_stripe(const StripeDesc* st, uint32_t n, uint32_t tile) {
  uint32_t lo = 0, hi = n;  // last stripe with tile_begin <= tile
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (st[mid].tile_begin <= tile) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The per-tile operation fields a body needs, held in registers.
struct TileOp {
  uint64_t read_mask;
  uint64_t pmask;
  int k, n_pos, e, m, op;
};

__device__ __forceinline__ void wait_or_fail(uint64_t* bar, uint32_t par, bool& failed, int* status, int code,
                                             unsigned long long limit) {
  if (!failed && !mbar_wait(bar, par, limit)) {
    failed = true;
    record_status(status, code);
  }
}

// The last n < 16 bytes of a block, read from global memory as a zero-padded
// 16-byte chunk.  A rolled loop: the path is cold (one chunk per block at
// most) and is instantiated at every unrolled input load, so it is kept
// small to leave the instruction cache to the arithmetic.
__device__ __forceinline__ uint4 ragged_load(const uint8_t* g, uint32_t n) {
  uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
#pragma unroll 1
  for (int t = (int)n - 1; t >= 0; --t) {
    w3 = (w3 << 8) | (w2 >> 24);
    w2 = (w2 << 8) | (w1 >> 24);
    w1 = (w1 << 8) | (w0 >> 24);
    w0 = (w0 << 8) | g[t];
  }
  return make_uint4(w0, w1, w2, w3);
}

// Store the first n < 16 bytes of a chunk (the ragged end of a block).
__device__ __forceinline__ void ragged_store(uint8_t* g, uint4 v, uint32_t n) {
  uint32_t a = v.x, b = v.y, c = v.z, d = v.w;
#pragma unroll 1
  for (uint32_t t = 0; t < n; ++t) {
    g[t] = (uint8_t)a;
    a = (a >> 8) | (b << 24);
    b = (b >> 8) | (c << 24);
    c = (c >> 8) | (d << 24);
    d >>= 8;
  }
}

// outp[t] for a runtime t without indexing the register array (which would
// put it in local memory); folds to outp[t] when t is a constant.
template <int MO>
__device__ __forceinline__ uint64_t select_out(const uint64_t (&outp)[MO], int t) {
  uint64_t p = outp[0];
#pragma unroll
  for (int u = 1; u < MO; ++u) p = (t == u) ? outp[u] : p;
  return p;
}

// ------------------------------------------------------ consumer tile views
// G column groups per lane: lane l owns the 16-byte chunks at
// l*16 + c*512 (c < G*W/4) of its warp's segment (G * segment_bytes(W)
// bytes); group g is words g*W .. g*W+W-1 of a load or store.
template <int W, int MO, int G = 1>
struct SymTile {
  Ring* ring;
  const uint64_t* ptrs;  // stripe pointers: inputs then outputs
  uint64_t outp[MO];     // output pointers, loaded at tile start
  int n_in;
  uint64_t goff;   // byte offset of the tile within each block
  uint32_t len;    // valid bytes of this tile (<= slice)
  uint32_t seg;    // this warp's segment offset
  uint32_t lane;
  int* status;
  unsigned long long limit;
  bool failed;
  bool whole;      // this thread's chunks are all full 16-byte chunks in the slot

  __device__ __forceinline__ void begin(const TileHeader& h) {
    ptrs = reinterpret_cast<const uint64_t*>(h.ptrs);
    n_in = h.n_in;
    goff = h.goff;
    len = h.len;
    // every chunk of this thread lies in the bulk-copied part of the slot
    whole = seg + (uint32_t)(G * W / 4 - 1) * 512u + lane * 16u + 16u <= (len & ~15u);
#pragma unroll
    for (int t = 0; t < MO; ++t) outp[t] = h.outp[t];
  }

  // Inputs are consumed in order 0..n_in-1, one ring slot each.
  __device__ __forceinline__ void load(int i, uint32_t* x) {
    Ring& r = *ring;
    const uint32_t s = r.s, par = r.par;
    r.advance();
    wait_or_fail(&r.full[s], par, failed, status, kDevErrTimeoutFull, limit);
    // After a timed-out wait the slot may hold stale bytes; they are read
    // anyway (the addresses are valid) and store() writes nothing.
    const uint8_t* slot = r.slots + (size_t)s * r.stride;
    if (whole) {
#pragma unroll
      for (int c = 0; c < G * W / 4; ++c) {
        const uint4 v = *reinterpret_cast<const uint4*>(slot + seg + (uint32_t)c * 512u + lane * 16u);
        x[4 * c + 0] = v.x;
        x[4 * c + 1] = v.y;
        x[4 * c + 2] = v.z;
        x[4 * c + 3] = v.w;
      }
    } else {
      const uint32_t len16 = len & ~15u;
#pragma unroll
      for (int c = 0; c < G * W / 4; ++c) {
        const uint32_t co = seg + (uint32_t)c * 512u + lane * 16u;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (co + 16u <= len16) {
          v = *reinterpret_cast<const uint4*>(slot + co);
        } else if (co < len) {
          v = ragged_load(reinterpret_cast<const uint8_t*>(ptrs[i]) + goff + co, min(len - co, 16u));
        }
        x[4 * c + 0] = v.x;
        x[4 * c + 1] = v.y;
        x[4 * c + 2] = v.z;
        x[4 * c + 3] = v.w;
      }
    }
    mbar_arrive(&r.empty[s]);
  }

  __device__ __forceinline__ void store(int t, const uint32_t* x) {
    if (failed) return;
    uint8_t* out = reinterpret_cast<uint8_t*>(select_out(outp, t)) + goff;
    if (whole) {
#pragma unroll
      for (int c = 0; c < G * W / 4; ++c)
        *reinterpret_cast<uint4*>(out + seg + (uint32_t)c * 512u + lane * 16u) =
            make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
      return;
    }
#pragma unroll
    for (int c = 0; c < G * W / 4; ++c) {
      const uint32_t co = seg + (uint32_t)c * 512u + lane * 16u;
      const uint4 v = make_uint4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
      if (co + 16u <= len) {
        *reinterpret_cast<uint4*>(out + co) = v;
      } else if (co < len) {
        ragged_store(out + co, v, len - co);
      }
    }
  }
};

// Packet layout: thread `unit` (warp*32 + lane) owns unit `unit` of the tile
// (G adjacent 32-bit words of each of the W packet rows); group g of a load
// or store is words g*W .. g*W+W-1 (word g of each row).  Where the unit
// lies in the slot and in the block is worked out once per tile.
template <int W, int MO, int G = 1>
struct PacketTile {
  static_assert(G == 1 || G == 2, "one or two groups");
  static constexpr uint32_t kUnitBytes = 4u * G;
  Ring* ring;
  const uint64_t* ptrs;
  uint64_t outp[MO];  // output pointers, loaded at tile start
  int n_in;
  uint64_t gbase;     // byte offset of this unit's row 0 in a block
  uint32_t sbase;     // byte offset of this unit's row 0 in a slot
  uint32_t srow;      // slot bytes between packet rows of this unit
  uint32_t P;         // packet bytes (block bytes between packet rows)
  uint32_t unit;      // this thread's unit inside the tile
  bool valid;         // the unit exists (the last tile of a block may be short)
  bool whole_sp;      // the slot holds whole super-packets (JobParams::packet_whole)
  int* status;
  unsigned long long limit;
  bool failed;

  __device__ __forceinline__ void begin(const TileHeader& h) {
    ptrs = reinterpret_cast<const uint64_t*>(h.ptrs);
    n_in = h.n_in;
    P = h.packet_bytes;
#pragma unroll
    for (int t = 0; t < MO; ++t) outp[t] = h.outp[t];
    const UnitPlace u = packet_unit_place<W, G>(h.goff, h.len, h.col0, h.head, h.whole, P, whole_sp, unit);
    valid = u.valid;
    sbase = u.sbase;
    srow = u.srow;
    gbase = u.gbase;
  }

  __device__ __forceinline__ void load(int i, uint32_t* x) {
    Ring& r = *ring;
    const uint32_t s = r.s, par = r.par;
    r.advance();
    wait_or_fail(&r.full[s], par, failed, status, kDevErrTimeoutFull, limit);
    const uint8_t* slot = r.slots + (size_t)s * r.stride + sbase;
    // stale after a timed-out wait; store() then writes nothing
    if constexpr (G == 1) {
#pragma unroll
      for (int c = 0; c < W; ++c) x[c] = *reinterpret_cast<const uint32_t*>(slot + c * srow);
    } else {
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const uint2 v = *reinterpret_cast<const uint2*>(slot + c * srow);
        x[c] = v.x;
        x[W + c] = v.y;
      }
    }
    mbar_arrive(&r.empty[s]);
  }

  __device__ __forceinline__ void store(int t, const uint32_t* x) {
    if (failed || !valid) return;
    uint8_t* out = reinterpret_cast<uint8_t*>(select_out(outp, t)) + gbase;
    if constexpr (G == 1) {
#pragma unroll
      for (int c = 0; c < W; ++c) *reinterpret_cast<uint32_t*>(out + (size_t)c * P) = x[c];
    } else {
#pragma unroll
      for (int c = 0; c < W; ++c) *reinterpret_cast<uint2*>(out + (size_t)c * P) = make_uint2(x[c], x[W + c]);
    }
  }
};

// Runtime decode matrix W in selector form (Selectors<W, M> layout).
struct CoefWords {
  const uint32_t* base;
  __device__ __forceinline__ uint32_t word(int i) const { return base[i]; }
};

// Runtime parity matrix P: column j as packed bits (PackedBits<W, M, 1>),
// column_words(M, W) words per column.
template <int W, int M>
struct ColumnWords {
  const uint32_t* base;
  struct Column {
    const uint32_t* p;
    __device__ __forceinline__ uint32_t word(int i) const { return p[i]; }
  };
  __device__ __forceinline__ Column column(int j) const { return Column{base + j * ((M * W + 31) / 32)}; }
};

// ------------------------------------------------------------------ bodies
// Register split: the producer gets a warpgroup of its own (4 warps, one of
// them working) that gives back registers with setmaxnreg.dec, and the
// consumer warpgroups take them with setmaxnreg.inc.  A CTA of 4 + NC warps
// is launched at the registers a thread its size allows (128 for 4 + 12
// warps: the 64K of an SM; 168 for 4 + 8); the producer warpgroup drops to
// P, the NC consumer warps rise to C, with 128 P + 32 NC C at most the
// launch's registers, so every launch of fewer consumer warps fits too (the
// shares are checked against the compiled count before the first launch).
// Used where the extra registers were measured to pay: the two-group
// decodes with pair sums in the decode-matrix step, the GF(2^16) decodes
// (12 instead of 8 consumer warps) and the GF(2^16) two-group packet
// encode.  The packet-layout producer needs more registers than the
// symbol-layout one.
constexpr int kSplitMaxConsumers = 12;
// registers a thread at launch for a CTA of `threads` threads (warps take
// registers in groups of four, a thread's count is a multiple of 8)
RS_CHD constexpr int launch_regs(int threads) { return 65536 / ((threads + 127) / 128 * 128) / 8 * 8; }
template <int P, int C, int NC = kSplitMaxConsumers>
struct RegSplit {
  static_assert(NC % 4 == 0 && P % 8 == 0 && C % 8 == 0 && C <= 256 &&
                    P * 128 + C * 32 * NC <= launch_regs((NC + 4) * 32) * (NC + 4) * 32,
                "register split exceeds the launch's registers");
  static constexpr int kProducerWarps = 4;
  static constexpr int kProducerRegs = P;
  static constexpr int kConsumerRegs = C;
  static constexpr int kSplitConsumers = NC;
};
struct NoSplit {
  static constexpr int kProducerWarps = 1;
  static constexpr int kProducerRegs = 0;
  static constexpr int kConsumerRegs = 0;
};
using SymbolDecodeSplit = RegSplit<56, 152>;  // two-group symbol-layout decode, pair sums
using PacketDecodeSplit = RegSplit<80, 144>;  // two-group packet-layout decode, pair sums
using Wide16DecodeSplit = RegSplit<104, 136>; // GF(2^16) one-group decodes
using Packet16Encode2Split = RegSplit<96, 200, 8>;  // GF(2^16) two-group packet encode and decode

RS_CHD constexpr int body_warps(int regs_words) { return regs_words <= 48 ? 16 : 8; }
// Register budget: 8-warp GF(2^8) bodies whose live state (accumulators,
// plus the outputs for a decode) is at most 64 words are compiled for two
// resident CTAs per SM (about 113 registers), which they fit without
// spilling; the others keep the one-CTA budget.
RS_CHD constexpr int body_min_blocks(int w, int max_warps, int live_words) {
  return (w == 8 && max_warps <= 8 && live_words <= 64) ? 2 : 1;
}

// One-group GF(2^8) decodes that keep more than four syndromes (two
// selector chunks, 122-141 registers at m = 5, 6) get 12 consumer warps
// from the split instead of 8.
template <int W, int M, int OP>
using PolyBodySplit =
    std::conditional_t<OP == kOpDecode && W == 16, Wide16DecodeSplit,
                       std::conditional_t<OP == kOpDecode && W == 8 && (M == 5 || M == 6), SymbolDecodeSplit, NoSplit>>;

template <int W, int M, int OP>
struct PolyBody : PolyBodySplit<W, M, OP> {
  static constexpr int kW = W;
  static constexpr int kGroups = 1;
  static constexpr int kLayout = kLayoutSymbol;
  static constexpr int kMaxOut = M;
  static constexpr int kMaxWarps =
      PolyBody::kProducerWarps == 4 ? kSplitMaxConsumers : (OP == kOpEncode ? body_warps(M * W) : 8);
  static constexpr int kMinBlocks =
      PolyBody::kProducerWarps == 4 ? 1 : body_min_blocks(W, kMaxWarps, (OP == kOpEncode ? 1 : 2) * M * W);
  __device__ static bool matches(const TileOp& o) { return o.op == OP && o.m == M; }
  template <class Tile>
  __device__ static void run(const TileOp& o, Tile& t, const uint32_t* coef) {
    if constexpr (OP == kOpEncode) {
      PolyEncode<W, M>::run(o.k, t, t);
    } else {
      CoefWords cm{coef};
      PolyDecode<W, M>::run(o.n_pos, o.read_mask, o.e, t, t, cm);
    }
  }
};

// Compile-time-P encode with two 32-column groups per lane: MatEncodeFixed2.
// Symbol layout (GF(2^8), M <= 4): 12 warps at 128 registers.  Packet
// layout over GF(2^16): the 2 x M x 16 accumulator planes need the register
// split's 200 registers, 8 consumer warps; a tile of 8 x 32 units of two
// words is then one whole super-packet of 2 KiB packets, fetched by one
// bulk copy per block (the one-group kernel's 480-unit tiles straddle the
// 512-unit super-packets).
template <int W, int K, int M, int KIND>
struct MatFixedEncode2Body
    : std::conditional_t<kind_layout(KIND) == kLayoutPacket, Packet16Encode2Split, NoSplit> {
  static constexpr int kW = W;
  static constexpr int kGroups = 2;
  static constexpr int kLayout = kind_layout(KIND);
  static constexpr int kMaxOut = M;
  static constexpr int kMaxWarps = kLayout == kLayoutPacket ? Packet16Encode2Split::kSplitConsumers : 12;
  static constexpr int kMinBlocks = 1;
  static_assert(kLayout == kLayoutSymbol || W == 16, "packet layout: GF(2^16) only");
  __device__ static bool matches(const TileOp& o) { return o.op == kOpMatEncode && o.m == M && o.k == K; }
  template <class Tile>
  __device__ static void run(const TileOp&, Tile& t, const uint32_t*) {
    MatEncodeFixed2<W, K, M, KIND, kLayout == kLayoutSymbol>::run(t, t);
  }
};

// GF(2^8) polynomial decode with two 32-column groups per lane
// (PolyDecode2): 64 columns per thread share every warp-uniform decision.
template <int W, int M>
struct PolyDecode2Body : SymbolDecodeSplit {
  static constexpr int kW = W;
  static constexpr int kGroups = 2;
  static constexpr int kLayout = kLayoutSymbol;
  static constexpr int kMaxOut = M;
  // two groups of syndromes and outputs live at once, plus the pair sums
  // for m <= 4 (m = 5, 6: two selector chunks, no pair sums): 12 consumer
  // warps at the split's 152 registers
  static constexpr int kMaxWarps = kSplitMaxConsumers;
  static constexpr int kMinBlocks = 1;
  __device__ static bool matches(const TileOp& o) { return o.op == kOpDecode && o.m == M; }
  template <class Tile>
  __device__ static void run(const TileOp& o, Tile& t, const uint32_t* coef) {
    CoefWords cm{coef};
    PolyDecode2<W, M, (M <= 4)>::run(o.n_pos, o.read_mask, o.e, t, t, cm);
  }
};

template <int W, int M, int OP, int LAYOUT>
struct MatRuntimeBody : NoSplit {
  static constexpr int kW = W;
  static constexpr int kGroups = 1;
  static constexpr int kLayout = LAYOUT;
  static constexpr int kMaxOut = M;
  static constexpr int kMaxWarps = OP == kOpMatEncode ? body_warps(M * W + 16) : 8;
  static constexpr int kMinBlocks = body_min_blocks(W, kMaxWarps, (OP == kOpMatEncode ? 1 : 2) * M * W + 16);
  __device__ static bool matches(const TileOp& o) { return o.op == OP && o.m == M; }
  template <class Tile>
  __device__ static void run(const TileOp& o, Tile& t, const uint32_t* coef) {
    ColumnWords<W, M> cols{reinterpret_cast<const uint32_t*>(o.pmask)};
    if constexpr (OP == kOpMatEncode) {
      MatEncodeRuntime<W, M, LAYOUT == kLayoutSymbol>::run(o.k, t, t, cols);
    } else {
      CoefWords cm{coef};
      MatDecodeRuntime<W, M, LAYOUT == kLayoutSymbol>::run(o.k, o.read_mask, o.e, t, t, cols, cm);
    }
  }
};

template <int W, int K, int M, int KIND, int OP>
using MatFixedBodySplit = std::conditional_t<
    OP == kOpMatDecode && W == 16, Wide16DecodeSplit,
    std::conditional_t<OP == kOpMatDecode && W == 8 && (M == 5 || M == 6),
                       std::conditional_t<kind_layout(KIND) == kLayoutPacket, PacketDecodeSplit, SymbolDecodeSplit>,
                       NoSplit>>;

template <int W, int K, int M, int KIND, int OP>
struct MatFixedBody : MatFixedBodySplit<W, K, M, KIND, OP> {
  static constexpr int kW = W;
  static constexpr int kGroups = 1;
  static constexpr int kLayout = kind_layout(KIND);
  static constexpr int kMaxOut = M;
  // GF(2^16) packet-layout encodes (pure XOR networks, about 125
  // registers) may run 15 consumer warps at the 128-register cap
  static constexpr int kMaxWarps =
      MatFixedBody::kProducerWarps == 4
          ? kSplitMaxConsumers
          : (OP == kOpMatEncode ? (W == 16 && kind_layout(KIND) == kLayoutPacket ? 15 : body_warps(M * W)) : 8);
  static constexpr int kMinBlocks =
      MatFixedBody::kProducerWarps == 4 ? 1 : body_min_blocks(W, kMaxWarps, (OP == kOpMatEncode ? 1 : 2) * M * W);
  __device__ static bool matches(const TileOp& o) { return o.op == OP && o.m == M && o.k == K; }
  template <class Tile>
  __device__ static void run(const TileOp& o, Tile& t, const uint32_t* coef) {
    if constexpr (OP == kOpMatEncode) {
      MatEncodeFixed<W, K, M, KIND, kLayout == kLayoutSymbol>::run(t, t);
    } else {
      CoefWords cm{coef};
      MatDecodeFixed<W, K, M, KIND, kLayout == kLayoutSymbol>::run(o.read_mask, o.e, t, t, cm);
    }
  }
};

// Compile-time-P decode (M <= 4) with two 32-column groups per lane
// (MatDecodeFixed2), in either layout.
template <int W, int KIND>
using Decode2Split = std::conditional_t<kind_layout(KIND) == kLayoutPacket,
                                        std::conditional_t<W == 16, Packet16Encode2Split, PacketDecodeSplit>, NoSplit>;
template <int W, int K, int M, int KIND>
struct MatFixedDecode2Body : Decode2Split<W, KIND> {
  static constexpr int kW = W;
  static constexpr int kGroups = 2;
  static constexpr int kLayout = kind_layout(KIND);
  static constexpr int kMaxOut = M;
  // symbol layout: up to 15 warps at 128 registers (the pair sums measured
  // slower there: they spill at the split's budget); packet layout over
  // GF(2^8): the register split and pair sums, 12 warps at 144 registers;
  // over GF(2^16): 8 warps at 200 registers without pair sums (a tile of 256
  // two-word units is one super-packet of 2 KiB packets, as in the encode)
  static constexpr bool kPairSums = kLayout == kLayoutPacket && W == 8;
  static constexpr int kMaxWarps =
      kLayout == kLayoutSymbol ? 15 : (W == 16 ? Packet16Encode2Split::kSplitConsumers : kSplitMaxConsumers);
  static constexpr int kMinBlocks = 1;
  __device__ static bool matches(const TileOp& o) { return o.op == kOpMatDecode && o.m == M && o.k == K; }
  template <class Tile>
  __device__ static void run(const TileOp& o, Tile& t, const uint32_t* coef) {
    CoefWords cm{coef};
    MatDecodeFixed2<W, K, M, KIND, kLayout == kLayoutSymbol, kPairSums>::run(o.read_mask, o.e, t, t, cm);
  }
};

// Several bodies of the same width and layout in one kernel: each stripe
// runs the first body whose matches() accepts it.
template <class First, class... Rest>
struct MixedBody {
  static constexpr int kW = First::kW;
  static constexpr int kGroups = First::kGroups;
  static_assert(((Rest::kGroups == First::kGroups) && ...), "one tile geometry per kernel");
  static constexpr int kLayout = First::kLayout;
  static constexpr int min_warps() {
    int w = First::kMaxWarps;
    ((w = Rest::kMaxWarps < w ? Rest::kMaxWarps : w), ...);
    return w;
  }
  static constexpr int kMaxWarps = min_warps();
  static constexpr int max_out() {
    int o = First::kMaxOut;
    ((o = Rest::kMaxOut > o ? Rest::kMaxOut : o), ...);
    return o;
  }
  static constexpr int kMaxOut = max_out();
  static constexpr int min_blocks() {
    int b = First::kMinBlocks;
    ((b = Rest::kMinBlocks < b ? Rest::kMinBlocks : b), ...);
    return b;
  }
  static constexpr int kMinBlocks = min_blocks();
  static constexpr int kProducerWarps = First::kProducerWarps;
  static constexpr int kProducerRegs = First::kProducerRegs;
  static constexpr int kConsumerRegs = First::kConsumerRegs;
  static_assert(((Rest::kProducerWarps == First::kProducerWarps && Rest::kProducerRegs == First::kProducerRegs &&
                  Rest::kConsumerRegs == First::kConsumerRegs) && ...),
                "one warp layout per kernel");
  __device__ static bool matches(const TileOp& o) { return First::matches(o) || (Rest::matches(o) || ...); }
  template <class Tile>
  __device__ static void run(const TileOp& o, Tile& t, const uint32_t* coef) {
    if (First::matches(o)) {
      First::run(o, t, coef);
      return;
    }
    if constexpr (sizeof...(Rest) > 0) MixedBody<Rest...>::run(o, t, coef);
  }
};

// ---------------------------------------------------------------- producer
// The CTA's tiles: a contiguous run [begin, end) of the launch's tiles.
struct TileRange {
  uint32_t begin, end;
};
__device__ __forceinline__ TileRange cta_tiles(uint32_t total_tiles) {
  const uint32_t per = (total_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t b = min(blockIdx.x * per, total_tiles);
  return TileRange{b, min(b + per, total_tiles)};
}

template <int W, int LAYOUT, int G>
__device__ __forceinline__ void producer_loop(const JobParams& p, const StripeDesc* stripes, const uint64_t* ptrs,
                                              const uint32_t* coef, TileHeader* headers, Ring& ring,
                                              uint32_t n_stripes, uint32_t total_tiles) {
  if (p.inject == kInjectProducerStall && blockIdx.x == 0) return;  // test hook, see job.hpp
  const TileRange tr = cta_tiles(total_tiles);
  if (tr.begin >= tr.end) return;
  uint32_t q = 0;
  bool ok = true;
  // current stripe, held in registers; re-read only when a tile crosses into
  // the next stripe
  uint32_t si = find_stripe(stripes, n_stripes, tr.begin);
  StripeDesc d = stripes[si];
  uint32_t next_begin = si + 1 < n_stripes ? stripes[si + 1].tile_begin : total_tiles;
  bool fresh = true;      // header fields of this stripe not yet in shared memory
  uint32_t prev_h = 0;    // slot whose header holds this stripe's fields
  for (uint32_t tile = tr.begin; tile < tr.end && ok; ++tile) {
    while (tile >= next_begin) {
      ++si;
      d = stripes[si];
      next_begin = si + 1 < n_stripes ? stripes[si + 1].tile_begin : total_tiles;
      fresh = true;
    }
    const TileGeom g = tile_geom<G>(d, tile - d.tile_begin, ring.slice, W);
    const uint64_t* ip = ptrs + d.ptr_off;
    for (int i = 0; i < d.n_in; ++i) {
      const uint32_t s = ring.s, par = ring.par;
      if (q >= ring.depth && !mbar_wait(&ring.empty[s], par ^ 1u, p.wait_limit_ns)) {
        record_status(p.status, kDevErrTimeoutEmpty);
        ok = false;
        break;
      }
      if (i == 0) {
        // the tile's header travels with its first slot
        TileHeader& h = headers[s];
        h.goff = g.goff;
        h.len = g.len;
        h.col0 = g.col0;
        h.head = g.head;
        h.whole = g.whole;
        h.read_mask = d.read_mask;
        h.pmask = d.pmask;
        h.ptrs = reinterpret_cast<uint64_t>(ip);
        h.packet_bytes = d.packet_bytes;
        h.n_in = d.n_in;
        h.n_out = d.n_out;
        h.op = d.op;
        h.m = d.m;
        h.k = d.k;
        h.n_pos = d.n_pos;
        h.e = d.e;
        const bool dec = d.op == kOpDecode || d.op == kOpMatDecode;
        const int words = dec ? selector_words((int)d.m, W) : 0;
        if (fresh) {
          for (int t = 0; t < kMaxM; ++t) h.outp[t] = t < (int)d.n_out ? ip[d.n_in + t] : 0ull;
          for (int c = 0; c < words; ++c) h.coef[c] = coef[d.coef_off + c];
          fresh = false;
        } else if (prev_h != s) {
          // same stripe: output pointers and coefficients from the previous
          // tile's header (no other header is written in between)
          const TileHeader& o = headers[prev_h];
          for (int t = 0; t < kMaxM; ++t) h.outp[t] = o.outp[t];
          for (int c = 0; c < words; ++c) h.coef[c] = o.coef[c];
        }
        prev_h = s;
      }
      uint8_t* dst = ring.slots + (size_t)s * ring.stride;
      const uint8_t* src = reinterpret_cast<const uint8_t*>(ip[i]) + g.goff;
      if constexpr (LAYOUT == kLayoutSymbol) {
        const uint32_t len16 = g.len & ~15u;
        if (len16) {
          mbar_arrive_expect_tx(&ring.full[s], len16);
          tma_load_1d(dst, src, len16, &ring.full[s]);
        } else {
          mbar_arrive(&ring.full[s]);
        }
      } else {
        uint64_t* full = &ring.full[s];
        packet_copies<W, G>(
            g, d.packet_bytes, p.packet_whole != 0, [full](uint32_t bytes) { mbar_arrive_expect_tx(full, bytes); },
            [dst, src, full](uint32_t so, uint32_t go, uint32_t n) { tma_load_1d(dst + so, src + go, n, full); });
      }
      ring.advance();
      ++q;
    }
  }
  // Drain: the CTA must not retire with bulk copies still writing its shared
  // memory, so wait for the last fills to land (they complete on their own).
  const uint32_t first = q > ring.depth ? q - ring.depth : 0;
  for (uint32_t f = first; f < q; ++f) {
    if (!mbar_wait(&ring.full[f % ring.depth], (f / ring.depth) & 1u, p.wait_limit_ns))
      record_status(p.status, kDevErrTimeoutDrain);
  }
}

// ------------------------------------------------------------------ kernel
template <class Body>
RS_CHD constexpr int body_threads() {
  return (Body::kMaxWarps + Body::kProducerWarps) * 32;
}

template <class Body>
__global__ void __launch_bounds__(body_threads<Body>(), Body::kMinBlocks)
    rs_stripe_kernel(const __grid_constant__ JobParams p) {
  constexpr int W = Body::kW;
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t depth = p.depth;
  Ring ring;
  ring.full = reinterpret_cast<uint64_t*>(smem);
  ring.empty = ring.full + depth;
  TileHeader* headers = reinterpret_cast<TileHeader*>(smem + ((2u * depth * 8u + 127u) & ~127u));
  ring.slots = reinterpret_cast<uint8_t*>(headers) + (size_t)depth * kHeaderBytes;
  ring.depth = depth;
  ring.slice = p.slice_bytes;
  ring.stride = p.slot_bytes ? p.slot_bytes : p.slice_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // consumer warps 0..nc-1, then the producer warp (or warpgroup)
  const int nc = (int)(blockDim.x >> 5) - Body::kProducerWarps;
  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < depth; ++s) {
      mbar_init(&ring.full[s], 1);
      mbar_init(&ring.empty[s], (uint32_t)nc * 32u);
    }
    fence_barrier_init();
  }
  __syncthreads();
  const StripeDesc* stripes = p.stripes ? p.stripes : &p.inl_stripe;
  const uint64_t* ptrs = p.ptrs ? p.ptrs : p.inl_ptrs;
  const uint32_t* coef = p.coef ? p.coef : p.inl_coef;
  const uint32_t n_stripes = p.counts ? p.counts[0] : p.n_stripes;
  const uint32_t total_tiles = p.counts ? p.counts[1] : p.total_tiles;

  if (warp >= nc) {
    if constexpr (Body::kProducerWarps == 4) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(Body::kProducerRegs));
    if (warp == nc && lane == 0)
      producer_loop<W, Body::kLayout, Body::kGroups>(p, stripes, ptrs, coef, headers, ring, n_stripes, total_tiles);
    return;
  }
  if constexpr (Body::kProducerWarps == 4) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(Body::kConsumerRegs));

  using Tile = std::conditional_t<Body::kLayout == kLayoutSymbol, SymTile<W, Body::kMaxOut, Body::kGroups>,
                                  PacketTile<W, Body::kMaxOut, Body::kGroups>>;
  Tile tile;
  tile.ring = &ring;
  tile.status = p.status;
  tile.limit = p.wait_limit_ns;
  tile.failed = false;
  if constexpr (Body::kLayout == kLayoutSymbol) {
    tile.lane = (uint32_t)lane;
    tile.seg = (uint32_t)warp * (uint32_t)Body::kGroups * segment_bytes(W);
  } else {
    tile.unit = (uint32_t)(warp * 32 + lane);
    tile.whole_sp = p.packet_whole != 0;
  }
  const TileRange tr = cta_tiles(total_tiles);
  for (uint32_t t = tr.begin; t < tr.end; ++t) {
    // the tile's header is published by its first slot's full barrier
    wait_or_fail(&ring.full[ring.s], ring.par, tile.failed, p.status, kDevErrTimeoutFull, p.wait_limit_ns);
    if (tile.failed) break;
    const TileHeader& h = headers[ring.s];
    const TileOp op{h.read_mask, h.pmask, (int)h.k, (int)h.n_pos, (int)h.e, (int)h.m, (int)h.op};
    tile.begin(h);
    Body::run(op, tile, h.coef);  // bodies read h.coef before releasing the slot
    if (tile.failed) break;
  }
}

// Launch one instantiation (sets the shared-memory attribute once per device).
template <class Body>
cudaError_t launch_body(const JobParams& p, const LaunchShape& sh, cudaStream_t st) {
  constexpr int kMaxDevices = 64;
  static std::once_flag once[kMaxDevices];
  static cudaError_t attr_err[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (sh.threads > body_threads<Body>() || sh.threads % 32 || sh.threads / 32 <= Body::kProducerWarps)
    return cudaErrorInvalidConfiguration;
  if constexpr (Body::kProducerWarps == 4) {
    // the producer warpgroup must start on a warpgroup boundary
    if ((sh.threads / 32 - 4) % 4) return cudaErrorInvalidConfiguration;
  }
  std::call_once(once[dev], [&] {
    attr_err[dev] = cudaFuncSetAttribute(rs_stripe_kernel<Body>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxDynamicSmem);
    if constexpr (Body::kProducerWarps == 4) {
      // setmaxnreg.inc draws on the registers the block was launched with:
      // check that the compiled count covers the split (a shortfall would
      // leave the consumers waiting for registers that never come)
      cudaFuncAttributes fa;
      cudaError_t e2 = cudaFuncGetAttributes(&fa, rs_stripe_kernel<Body>);
      if (e2 == cudaSuccess && fa.numRegs * body_threads<Body>() <
                                   Body::kProducerRegs * 128 + Body::kConsumerRegs * 32 * Body::kMaxWarps)
        e2 = cudaErrorInvalidConfiguration;
      if (attr_err[dev] == cudaSuccess) attr_err[dev] = e2;
    }
  });
  if (attr_err[dev] != cudaSuccess) return attr_err[dev];
  rs_stripe_kernel<Body><<<sh.grid, sh.threads, sh.smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace rsgb
