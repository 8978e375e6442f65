// Work description shared by the host planner and the kernels.
//
// A launch processes a list of stripe operations.  Every stripe is cut into
// tiles of `slice_bytes` per block; tiles of all stripes are numbered
// globally and CTAs take them round-robin.  For each tile the producer
// streams one slice per input block (in the codec's consumption order)
// through the shared-memory ring; consumers turn the slices into output
// slices written straight to HBM.
#pragma once
#include <stdint.h>

#include "gf.hpp"

namespace rsgb {

enum : uint8_t {
  kOpEncode = 0,       // polynomial LFSR encode: inputs d_{k-1}..d_0, outputs p_0..p_{m-1}
  kOpDecode = 1,       // polynomial Horner-syndrome decode
  kOpMatEncode = 2,    // matrix realization encode (runtime coefficient masks)
  kOpMatDecode = 3,    // matrix realization decode through H = [P | I]
};

enum : uint8_t { kLayoutSymbol = 0, kLayoutPacket = 1 };

// Matrix realizations with a compile-time generator
enum : int { kKindVandermonde = 1, kKindCauchy = 2, kKindPolyMatrix = 3, kKindPolyBitMatrix = 4, kKindGoodCauchy = 5 };

// Layout of a matrix kind: the bit-matrix kinds keep §2.3's packet layout.
RS_CHD constexpr int kind_layout(int kind) {
  return (kind == kKindCauchy || kind == kKindPolyBitMatrix || kind == kKindGoodCauchy) ? 1 : 0;
}

struct StripeDesc {
  uint64_t bytes;       // block bytes B
  uint64_t read_mask;   // decode: bit p set = position / block p is read
  uint32_t tile_begin;  // first global tile index of this stripe
  uint32_t ptr_off;     // first pointer: n_in inputs, then n_out outputs
  uint32_t coef_off;    // coefficient masks (words) for runtime matrices
  uint16_t n_in;        // input blocks streamed per tile
  uint16_t n_out;       // output blocks written per tile
  uint8_t op;
  uint8_t m;            // encode: m; decode: syndromes M
  uint8_t n_pos;        // decode: codeword length n
  uint8_t e;            // decode: outputs
  uint8_t k;            // data blocks
  uint8_t layout;       // kLayoutSymbol / kLayoutPacket
  uint16_t pad;
  uint32_t packet_bytes;  // packet layout: P
  uint32_t pad2;
  uint64_t pmask;       // matrix realizations, runtime P: device table of
                        // column masks [j][i][c] (k x m x W words)
};

// Test hook: CTA 0's producer issues nothing, so that CTA's consumers run
// into the bounded wait, record the timeout and return (no copy is ever in
// flight for that CTA, so nothing is left writing its shared memory).
constexpr uint32_t kInjectProducerStall = 1;

constexpr int kMaxPtrs = kMaxBlocks + kMaxM;
constexpr int kMaxCoefWords = kMaxM * kMaxM * 16;

struct JobParams {
  const StripeDesc* stripes;  // device table, or nullptr for the inline stripe
  const uint64_t* ptrs;       // device table, or nullptr
  const uint32_t* coef;       // device table, or nullptr
  int* status;                // device status word (0 = ok), may be nullptr
  const uint32_t* counts;     // device {n_stripes, total_tiles}, or nullptr
  uint32_t n_stripes;
  uint32_t total_tiles;
  uint32_t slice_bytes;       // bytes of one block per tile
  uint32_t depth;             // ring slots
  unsigned long long wait_limit_ns;  // bound of every pipeline wait (0 = default 2 s)
  uint32_t inject;            // test hook: kInjectProducerStall
  uint32_t packet_whole;      // packet layout: copy the whole super-packets a tile touches
  uint32_t slot_bytes;        // ring slot stride (>= slice_bytes; 0 = slice_bytes)
  uint32_t pad_slot;
  // one stripe passed by value (single-stripe calls need no device tables)
  StripeDesc inl_stripe;
  uint64_t inl_ptrs[kMaxPtrs];
  uint32_t inl_coef[kMaxCoefWords];
};

// What the producer tells the consumers about a tile, written into shared
// memory next to the tile's first slot before that slot is armed (so the
// slot's full barrier publishes it).  Consumers copy what they need into
// registers before they release that slot.
constexpr int kHeaderCoefWords = selector_words(kMaxM, 16);
struct alignas(16) TileHeader {
  uint64_t goff;            // symbol: byte offset; packet: offset of the first super-packet
  uint64_t read_mask;
  uint64_t pmask;
  uint64_t ptrs;            // this stripe's pointer table (ragged-end reads)
  uint64_t outp[kMaxM];
  uint32_t len;             // symbol: bytes; packet: units
  uint32_t col0;            // packet: first unit's column in its super-packet
  uint32_t head, whole;     // packet: units of the leading partial super-packet, whole ones after it
  uint32_t packet_bytes;
  uint16_t n_in, n_out;
  uint8_t op, m, k, n_pos, e, pad[3];
  uint32_t coef[kHeaderCoefWords];
};
constexpr uint32_t kHeaderBytes = (uint32_t)((sizeof(TileHeader) + 127) / 128 * 128);

// Bytes of one warp segment (32 lanes x 32 symbols) in the symbol layout.
RS_CHD constexpr uint32_t segment_bytes(int w) { return 32u * 32u * (uint32_t)(w / 8); }

}  // namespace rsgb
