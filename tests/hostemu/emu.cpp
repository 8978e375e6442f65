// Test harness: runs the library's codec templates (codec_poly.hpp,
// bitslice.hpp) and host planner (plan.cpp) on the CPU, with the same
// 32-symbol chunk layout as the GPU kernels (warp segment of 32 lanes, lane l
// owning the 16-byte chunks at l*16 + c*512).  It checks the bit-sliced
// arithmetic and the decode plans against the oracle without a GPU.  It is
// not a CPU fallback: nothing in the library calls it.
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "codec_matrix.hpp"
#include "codec_poly.hpp"
#include "job.hpp"
#include "plan.hpp"
#include "tile_geom.hpp"

using namespace rsgb;

namespace {

template <int W>
struct HostTile {
  const uint8_t* const* in;  // inputs in consumption order
  uint8_t* const* out;
  size_t B;
  size_t seg;   // segment offset within the block
  int lane;
  void load(int i, uint32_t* x) {
    for (int c = 0; c < W / 4; ++c) {
      const size_t co = seg + (size_t)c * 512 + (size_t)lane * 16;
      uint8_t b[16] = {0};
      for (int t = 0; t < 16; ++t)
        if (co + t < B) b[t] = in[i][co + t];
      for (int q = 0; q < 4; ++q)
        x[4 * c + q] = b[4 * q] | (b[4 * q + 1] << 8) | (b[4 * q + 2] << 16) | ((uint32_t)b[4 * q + 3] << 24);
    }
  }
  void store(int t, const uint32_t* x) {
    for (int c = 0; c < W / 4; ++c) {
      const size_t co = seg + (size_t)c * 512 + (size_t)lane * 16;
      for (int q = 0; q < 16; ++q)
        if (co + q < B) out[t][co + q] = (uint8_t)(x[4 * c + q / 4] >> (8 * (q % 4)));
    }
  }
};

// G column groups per lane: lane l owns the 16-byte chunks at
// l*16 + c*512 (c < G*W/4) of a segment of G*segment_bytes(W) bytes; group g
// is words g*W .. g*W+W-1 (chunks g*W/4 ..), as the device's G-group tiles.
template <int W, int G>
struct HostTileG {
  const uint8_t* const* in;
  uint8_t* const* out;
  size_t B;
  size_t seg;
  int lane;
  void load(int i, uint32_t* x) {
    for (int c = 0; c < G * W / 4; ++c) {
      const size_t co = seg + (size_t)c * 512 + (size_t)lane * 16;
      uint8_t b[16] = {0};
      for (int t = 0; t < 16; ++t)
        if (co + t < B) b[t] = in[i][co + t];
      for (int q = 0; q < 4; ++q)
        x[4 * c + q] = b[4 * q] | (b[4 * q + 1] << 8) | (b[4 * q + 2] << 16) | ((uint32_t)b[4 * q + 3] << 24);
    }
  }
  void store(int t, const uint32_t* x) {
    for (int c = 0; c < G * W / 4; ++c) {
      const size_t co = seg + (size_t)c * 512 + (size_t)lane * 16;
      for (int q = 0; q < 16; ++q)
        if (co + q < B) out[t][co + q] = (uint8_t)(x[4 * c + q / 4] >> (8 * (q % 4)));
    }
  }
};

struct HostCoef {
  std::vector<uint32_t> words;
  explicit HostCoef(const DecodePlan* pl, int w) : words(pack_decode_selectors(*pl, w)) {}
  uint32_t word(int i) const { return words[i]; }
};

template <int W, int M>
void run_encode(int k, uint8_t* blocks, size_t B) {
  std::vector<const uint8_t*> in(k);
  std::vector<uint8_t*> out(M);
  for (int i = 0; i < k; ++i) in[i] = blocks + (size_t)(k - 1 - i) * B;
  for (int j = 0; j < M; ++j) out[j] = blocks + (size_t)(k + j) * B;
  const size_t segb = segment_bytes(W);
  for (size_t seg = 0; seg < B; seg += segb)
    for (int lane = 0; lane < 32; ++lane) {
      HostTile<W> t{in.data(), out.data(), B, seg, lane};
      PolyEncode<W, M>::run(k, t, t);
    }
}

template <int W, int M>
void run_decode(const DecodePlan& pl, uint8_t* blocks, size_t B) {
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  for (int b : pl.in_blocks) in.push_back(blocks + (size_t)b * B);
  for (int b : pl.out_blocks) out.push_back(blocks + (size_t)b * B);
  const size_t segb = segment_bytes(W);
  HostCoef cf(&pl, W);
  for (size_t seg = 0; seg < B; seg += segb)
    for (int lane = 0; lane < 32; ++lane) {
      HostTile<W> t{in.data(), out.data(), B, seg, lane};
      PolyDecode<W, M>::run(pl.n_pos, pl.read_mask, pl.e, t, t, cf);
    }
}

template <int W, int M>
void run_decode2(const DecodePlan& pl, uint8_t* blocks, size_t B) {
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  for (int b : pl.in_blocks) in.push_back(blocks + (size_t)b * B);
  for (int b : pl.out_blocks) out.push_back(blocks + (size_t)b * B);
  const size_t segb = 2 * segment_bytes(W);
  HostCoef cf(&pl, W);
  for (size_t seg = 0; seg < B; seg += segb)
    for (int lane = 0; lane < 32; ++lane) {
      HostTileG<W, 2> t{in.data(), out.data(), B, seg, lane};
      PolyDecode2<W, M, (M <= 4)>::run(pl.n_pos, pl.read_mask, pl.e, t, t, cf);  // pair sums for M <= 4, as the kernel
    }
}

template <int W>
int encode_w(int k, int m, uint8_t* blocks, size_t B) {
  switch (m) {
    case 1: run_encode<W, 1>(k, blocks, B); return 0;
    case 2: run_encode<W, 2>(k, blocks, B); return 0;
    case 3: run_encode<W, 3>(k, blocks, B); return 0;
    case 4: run_encode<W, 4>(k, blocks, B); return 0;
    case 5: run_encode<W, 5>(k, blocks, B); return 0;
    case 6: run_encode<W, 6>(k, blocks, B); return 0;
    case 7: run_encode<W, 7>(k, blocks, B); return 0;
    case 8: run_encode<W, 8>(k, blocks, B); return 0;
  }
  return -1;
}

template <int W>
int decode_w(const DecodePlan& pl, uint8_t* blocks, size_t B) {
  switch (pl.M) {
    case 1: run_decode<W, 1>(pl, blocks, B); return 0;
    case 2: run_decode<W, 2>(pl, blocks, B); return 0;
    case 3: run_decode<W, 3>(pl, blocks, B); return 0;
    case 4: run_decode<W, 4>(pl, blocks, B); return 0;
    case 5: run_decode<W, 5>(pl, blocks, B); return 0;
    case 6: run_decode<W, 6>(pl, blocks, B); return 0;
    case 7: run_decode<W, 7>(pl, blocks, B); return 0;
    case 8: run_decode<W, 8>(pl, blocks, B); return 0;
  }
  return -1;
}

// Packet layout: the thread's W words are word u of the W packets of one
// super-packet.
template <int W>
struct HostPacketTile {
  const uint8_t* const* in;
  uint8_t* const* out;
  size_t sp_off;
  size_t P;
  size_t u;
  void load(int i, uint32_t* x) {
    for (int c = 0; c < W; ++c) {
      const uint8_t* p = in[i] + sp_off + (size_t)c * P + 4 * u;
      x[c] = p[0] | (p[1] << 8) | (p[2] << 16) | ((uint32_t)p[3] << 24);
    }
  }
  void store(int t, const uint32_t* x) {
    for (int c = 0; c < W; ++c) {
      uint8_t* p = out[t] + sp_off + (size_t)c * P + 4 * u;
      for (int q = 0; q < 4; ++q) p[q] = (uint8_t)(x[c] >> (8 * q));
    }
  }
};

template <int W, int M>
struct HostCols {
  std::vector<uint32_t> words;
  HostCols(const std::vector<uint32_t>& P, int k) : words(pack_columns(P, k, M, W)) {}
  struct Column {
    const uint32_t* p;
    uint32_t word(int i) const { return p[i]; }
  };
  Column column(int j) const { return Column{words.data() + (size_t)j * column_words(M, W)}; }
};

// Runs `body(tile)` over every 32-column group of the stripe in the layout.
template <int W, bool kPacket, class F>
void for_groups(const std::vector<const uint8_t*>& in, const std::vector<uint8_t*>& out, size_t B, size_t P, F&& body) {
  if (kPacket) {
    for (size_t sp = 0; sp < B; sp += (size_t)W * P)
      for (size_t u = 0; u < P / 4; ++u) {
        HostPacketTile<W> t{in.data(), out.data(), sp, P, u};
        body(t);
      }
  } else {
    const size_t segb = segment_bytes(W);
    for (size_t seg = 0; seg < B; seg += segb)
      for (int lane = 0; lane < 32; ++lane) {
        HostTile<W> t{in.data(), out.data(), B, seg, lane};
        body(t);
      }
  }
}

template <int W, int M, bool kPacket>
int mat_runtime(int k, const std::vector<uint32_t>& P, bool decode, const DecodePlan* pl, uint8_t* blocks, size_t B,
                size_t pkt) {
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  HostCols<W, M> cols(P, k);
  if (!decode) {
    for (int j = 0; j < k; ++j) in.push_back(blocks + (size_t)j * B);
    for (int i = 0; i < M; ++i) out.push_back(blocks + (size_t)(k + i) * B);
    for_groups<W, kPacket>(in, out, B, pkt, [&](auto& t) { MatEncodeRuntime<W, M, !kPacket>::run(k, t, t, cols); });
  } else {
    for (int b : pl->in_blocks) in.push_back(blocks + (size_t)b * B);
    for (int b : pl->out_blocks) out.push_back(blocks + (size_t)b * B);
    HostCoef cf(pl, W);
    for_groups<W, kPacket>(in, out, B, pkt, [&](auto& t) {
      MatDecodeRuntime<W, M, !kPacket>::run(k, pl->read_mask, pl->e, t, t, cols, cf);
    });
  }
  return 0;
}

template <int W, int K, int M, int KIND>
int mat_fixed(bool decode, const DecodePlan* pl, uint8_t* blocks, size_t B, size_t pkt) {
  constexpr bool kPacket = kind_layout(KIND) == 1;
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  if (!decode) {
    for (int j = 0; j < K; ++j) in.push_back(blocks + (size_t)j * B);
    for (int i = 0; i < M; ++i) out.push_back(blocks + (size_t)(K + i) * B);
    for_groups<W, kPacket>(in, out, B, pkt, [&](auto& t) { MatEncodeFixed<W, K, M, KIND, !kPacket>::run(t, t); });
  } else {
    for (int b : pl->in_blocks) in.push_back(blocks + (size_t)b * B);
    for (int b : pl->out_blocks) out.push_back(blocks + (size_t)b * B);
    HostCoef cf(pl, W);
    for_groups<W, kPacket>(in, out, B, pkt, [&](auto& t) {
      MatDecodeFixed<W, K, M, KIND, !kPacket>::run(pl->read_mask, pl->e, t, t, cf);
    });
  }
  return 0;
}

// The two-column-group compile-time-P decode (symbol layout).
template <int W, int K, int M, int KIND>
int mat_fixed2(const DecodePlan* pl, uint8_t* blocks, size_t B) {
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  for (int b : pl->in_blocks) in.push_back(blocks + (size_t)b * B);
  for (int b : pl->out_blocks) out.push_back(blocks + (size_t)b * B);
  HostCoef cf(pl, W);
  const size_t segb = 2 * segment_bytes(W);
  for (size_t seg = 0; seg < B; seg += segb)
    for (int lane = 0; lane < 32; ++lane) {
      HostTileG<W, 2> t{in.data(), out.data(), B, seg, lane};
      MatDecodeFixed2<W, K, M, KIND>::run(pl->read_mask, pl->e, t, t, cf);
    }
  return 0;
}

// Packet layout with two groups: the thread owns words 2u and 2u + 1 of the
// W packets of one super-packet; group g is word 2u + g of each packet.
template <int W>
struct HostPacketTile2 {
  const uint8_t* const* in;
  uint8_t* const* out;
  size_t sp_off;
  size_t P;
  size_t u;
  void load(int i, uint32_t* x) {
    for (int g = 0; g < 2; ++g)
      for (int c = 0; c < W; ++c) {
        const uint8_t* p = in[i] + sp_off + (size_t)c * P + 4 * (2 * u + g);
        x[g * W + c] = p[0] | (p[1] << 8) | (p[2] << 16) | ((uint32_t)p[3] << 24);
      }
  }
  void store(int t, const uint32_t* x) {
    for (int g = 0; g < 2; ++g)
      for (int c = 0; c < W; ++c) {
        uint8_t* p = out[t] + sp_off + (size_t)c * P + 4 * (2 * u + g);
        for (int q = 0; q < 4; ++q) p[q] = (uint8_t)(x[g * W + c] >> (8 * q));
      }
  }
};

// The two-column-group compile-time-P decode in the packet layout (pair
// sums over GF(2^8), none over GF(2^16), as the kernels).
template <int W, int K, int M, int KIND>
int mat_fixed2_packet(const DecodePlan* pl, uint8_t* blocks, size_t B, size_t P) {
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  for (int b : pl->in_blocks) in.push_back(blocks + (size_t)b * B);
  for (int b : pl->out_blocks) out.push_back(blocks + (size_t)b * B);
  HostCoef cf(pl, W);
  for (size_t sp = 0; sp < B; sp += (size_t)W * P)
    for (size_t u = 0; u < P / 8; ++u) {
      HostPacketTile2<W> t{in.data(), out.data(), sp, P, u};
      MatDecodeFixed2<W, K, M, KIND, false, W == 8>::run(pl->read_mask, pl->e, t, t, cf);
    }
  return 0;
}

// The two-column-group compile-time-P encode in the packet layout (the
// GF(2^16) kernel's body; no transposes).
template <int W, int K, int M, int KIND>
int mat_encode2_packet(uint8_t* blocks, size_t B, size_t P) {
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  for (int j = 0; j < K; ++j) in.push_back(blocks + (size_t)j * B);
  for (int i = 0; i < M; ++i) out.push_back(blocks + (size_t)(K + i) * B);
  for (size_t sp = 0; sp < B; sp += (size_t)W * P)
    for (size_t u = 0; u < P / 8; ++u) {
      HostPacketTile2<W> t{in.data(), out.data(), sp, P, u};
      MatEncodeFixed2<W, K, M, KIND, false>::run(t, t);
    }
  return 0;
}

template <int K, int M, int KIND>
int mat_encode2(uint8_t* blocks, size_t B) {
  std::vector<const uint8_t*> in;
  std::vector<uint8_t*> out;
  for (int j = 0; j < K; ++j) in.push_back(blocks + (size_t)j * B);
  for (int i = 0; i < M; ++i) out.push_back(blocks + (size_t)(K + i) * B);
  const size_t segb = 2 * segment_bytes(8);
  for (size_t seg = 0; seg < B; seg += segb)
    for (int lane = 0; lane < 32; ++lane) {
      HostTileG<8, 2> t{in.data(), out.data(), B, seg, lane};
      MatEncodeFixed2<8, K, M, KIND>::run(t, t);
    }
  return 0;
}

template <int W, bool kPacket>
int mat_runtime_m(int k, int m, const std::vector<uint32_t>& P, bool decode, const DecodePlan* pl, uint8_t* blocks,
                  size_t B, size_t pkt) {
  switch (m) {
    case 1: return mat_runtime<W, 1, kPacket>(k, P, decode, pl, blocks, B, pkt);
    case 2: return mat_runtime<W, 2, kPacket>(k, P, decode, pl, blocks, B, pkt);
    case 3: return mat_runtime<W, 3, kPacket>(k, P, decode, pl, blocks, B, pkt);
    case 4: return mat_runtime<W, 4, kPacket>(k, P, decode, pl, blocks, B, pkt);
    case 5: return mat_runtime<W, 5, kPacket>(k, P, decode, pl, blocks, B, pkt);
    case 6: return mat_runtime<W, 6, kPacket>(k, P, decode, pl, blocks, B, pkt);
    case 7: return mat_runtime<W, 7, kPacket>(k, P, decode, pl, blocks, B, pkt);
    case 8: return mat_runtime<W, 8, kPacket>(k, P, decode, pl, blocks, B, pkt);
  }
  return -1;
}

template <int KIND>
int mat_fixed_dispatch(int w, int k, int m, bool decode, const DecodePlan* pl, uint8_t* b, size_t B, size_t pkt) {
  if (KIND == 3 || KIND == 4) {
    if (w == 8 && k == 10 && m == 4) return mat_fixed<8, 10, 4, KIND>(decode, pl, b, B, pkt);
    if (w == 8 && k == 6 && m == 3) return mat_fixed<8, 6, 3, KIND>(decode, pl, b, B, pkt);
    if (w == 16 && k == 12 && m == 4) return mat_fixed<16, 12, 4, KIND>(decode, pl, b, B, pkt);
    return -2;
  }
  if (w == 8 && k == 6 && m == 3) return mat_fixed<8, 6, 3, KIND>(decode, pl, b, B, pkt);
  if (w == 8 && k == 10 && m == 4) return mat_fixed<8, 10, 4, KIND>(decode, pl, b, B, pkt);
  if (w == 8 && k == 12 && m == 4) return mat_fixed<8, 12, 4, KIND>(decode, pl, b, B, pkt);
  if (w == 8 && k == 20 && m == 4) return mat_fixed<8, 20, 4, KIND>(decode, pl, b, B, pkt);
  if (w == 16 && k == 12 && m == 4) return mat_fixed<16, 12, 4, KIND>(decode, pl, b, B, pkt);
  return -2;
}

}  // namespace

// The packet-layout tile geometry of the kernel (tile_geom.hpp) over a
// whole block: the producer's copies must stay inside the slot and the
// block and be 16-byte aligned, every valid unit's rows in the slot must
// hold the block bytes the unit stores to, and every unit of the block
// must be stored exactly once.  Returns the number of violations.
template <int W, int G>
long check_packet_tiles(uint32_t P, int nc, int nsp, bool whole_sp) {
  const uint32_t ub = 4u * G;
  const uint32_t slice = (uint32_t)nc * G * segment_bytes(W);
  const uint32_t wb = packet_whole_bytes(slice, W, G, P);
  const uint32_t slot = whole_sp ? (wb > slice ? wb : slice) : slice;
  const uint64_t B = (uint64_t)nsp * W * P;
  StripeDesc d{};
  d.layout = kLayoutPacket;
  d.bytes = B;
  d.packet_bytes = P;
  const uint32_t tiles = (uint32_t)((B + slice - 1) / slice);
  const uint32_t T = slice / (W * ub);
  std::vector<uint8_t> covered(B / ub, 0);
  long bad = 0;
  for (uint32_t lt = 0; lt < tiles; ++lt) {
    const TileGeom g = tile_geom<G>(d, lt, slice, W);
    std::vector<int64_t> src(slot / ub, -1);
    uint32_t total = 0;
    int armed = 0;
    packet_copies<W, G>(
        g, P, whole_sp,
        [&](uint32_t bytes) {
          total = bytes;
          ++armed;
        },
        [&](uint32_t so, uint32_t go, uint32_t n) {
          const uint64_t at = g.goff + go;
          if (armed != 1 || so % 16 || at % 16 || n % 16 || n == 0 || (uint64_t)so + n > slot || at + n > B) {
            ++bad;
            return;
          }
          for (uint32_t k = 0; k < n; k += ub) src[(so + k) / ub] = (int64_t)(at + k);
        });
    if (armed != 1) ++bad;
    uint64_t copied = 0;
    for (int64_t v : src) copied += v >= 0 ? ub : 0;
    if (copied != total) ++bad;
    for (uint32_t unit = 0; unit < T; ++unit) {
      const UnitPlace u = packet_unit_place<W, G>(g.goff, g.len, g.col0, g.head, g.whole, P, whole_sp, unit);
      if (u.valid != (unit < g.len)) ++bad;
      if (!u.valid) continue;
      for (int c = 0; c < W; ++c) {
        const uint64_t so = u.sbase + (uint64_t)c * u.srow, at = u.gbase + (uint64_t)c * P;
        if (so + ub > slot || at + ub > B || src[so / ub] != (int64_t)at || covered[at / ub]) {
          ++bad;
          continue;
        }
        covered[at / ub] = 1;
      }
    }
  }
  for (uint8_t c : covered) bad += c ? 0 : 1;
  return bad;
}

extern "C" {

// Packet tile geometry over one block of nsp super-packets (see
// check_packet_tiles); -1 for arguments the library rejects.
long emu_packet_tiles(int w, int groups, uint32_t P, int nc, int nsp, int whole_sp) {
  if (P == 0 || P % (128u * (uint32_t)groups) || nc < 1 || nc > 16 || nsp < 1) return -1;
  const bool ws = whole_sp != 0;
  if (w == 8 && groups == 1) return check_packet_tiles<8, 1>(P, nc, nsp, ws);
  if (w == 8 && groups == 2) return check_packet_tiles<8, 2>(P, nc, nsp, ws);
  if (w == 16 && groups == 1) return check_packet_tiles<16, 1>(P, nc, nsp, ws);
  return -1;
}


// Matrix realizations: kind 1 = Vandermonde (symbol layout), 2 = Cauchy
// (packet layout, packet bytes pkt), 3 = polynomial code as a matrix
// (symbol layout), 4 = its bit-matrix form (packet layout).  fixed:
// compile-time P kernels (only for the registered codes), else runtime P.
// er/e: decode when e > 0.
static bool host_parity(int w, int k, int m, int kind, std::vector<uint32_t>& P) {
  if (kind == 1) return vandermonde_parity_matrix(k, m, w, P);
  if (kind == 2) cauchy_parity_matrix(k, m, w, P);
  else if (kind == 5) good_cauchy_parity_matrix(k, m, w, P);
  else poly_parity_matrix(k, m, w, P);
  return true;
}

int emu_mat(int w, int k, int m, int kind, int fixed, const int* er, int e, int read_all, uint8_t* blocks, size_t B,
            size_t pkt) {
  std::vector<uint32_t> P;
  if (!host_parity(w, k, m, kind, P)) return -3;
  DecodePlan pl;
  const bool decode = e > 0;
  if (decode) {
    std::string err;
    if (!make_matrix_decode_plan(k, m, w, P, er, e, read_all != 0, pl, err)) return -1;
  }
  const DecodePlan* plp = decode ? &pl : nullptr;
  if (fixed) {
    switch (kind) {
      case 1: return mat_fixed_dispatch<1>(w, k, m, decode, plp, blocks, B, pkt);
      case 2: return mat_fixed_dispatch<2>(w, k, m, decode, plp, blocks, B, pkt);
      case 3: return mat_fixed_dispatch<3>(w, k, m, decode, plp, blocks, B, pkt);
      case 4: return mat_fixed_dispatch<4>(w, k, m, decode, plp, blocks, B, pkt);
      case 5: return mat_fixed_dispatch<5>(w, k, m, decode, plp, blocks, B, pkt);
    }
    return -2;
  }
  const bool packet = kind == 2 || kind == 4 || kind == 5;
  if (w == 8) return packet ? mat_runtime_m<8, true>(k, m, P, decode, plp, blocks, B, pkt)
                            : mat_runtime_m<8, false>(k, m, P, decode, plp, blocks, B, pkt);
  return packet ? mat_runtime_m<16, true>(k, m, P, decode, plp, blocks, B, pkt)
                : mat_runtime_m<16, false>(k, m, P, decode, plp, blocks, B, pkt);
}

// Two-column-group matrix decode (GF(2^8), symbol-layout kinds 1 and 3).
int emu_mat_decode2(int w, int k, int m, int kind, const int* er, int e, int read_all, uint8_t* blocks, size_t B) {
  if (w != 8 || (kind != 1 && kind != 3) || e <= 0) return -2;
  std::vector<uint32_t> P;
  if (!host_parity(w, k, m, kind, P)) return -3;
  DecodePlan pl;
  std::string err;
  if (!make_matrix_decode_plan(k, m, w, P, er, e, read_all != 0, pl, err)) return -1;
  if (pl.M > 4) return -2;
  if (kind == 1) {
    if (k == 10 && m == 4) return mat_fixed2<8, 10, 4, 1>(&pl, blocks, B);
    if (k == 6 && m == 3) return mat_fixed2<8, 6, 3, 1>(&pl, blocks, B);
    if (k == 20 && m == 4) return mat_fixed2<8, 20, 4, 1>(&pl, blocks, B);
  } else {
    if (k == 10 && m == 4) return mat_fixed2<8, 10, 4, 3>(&pl, blocks, B);
    if (k == 6 && m == 3) return mat_fixed2<8, 6, 3, 3>(&pl, blocks, B);
  }
  return -2;
}

// Two-column-group matrix decode in the packet layout (GF(2^8), kinds 2 and
// 4; P = packet bytes, a multiple of 8 dividing B / 8).
// The GF(2^16) two-group packet-layout encode (kinds 2 and 5, RS(12,4)).
int emu_mat_encode2_packet(int w, int k, int m, int kind, uint8_t* blocks, size_t B, size_t P) {
  if (w != 16 || k != 12 || m != 4 || P % 8 || B % (16 * P)) return -2;
  if (kind == 2) return mat_encode2_packet<16, 12, 4, 2>(blocks, B, P);
  if (kind == 5) return mat_encode2_packet<16, 12, 4, 5>(blocks, B, P);
  return -2;
}

int emu_mat_decode2_packet(int w, int k, int m, int kind, const int* er, int e, int read_all, uint8_t* blocks,
                           size_t B, size_t P) {
  if ((w != 8 && w != 16) || (kind != 2 && kind != 4 && kind != 5) || e <= 0 || P % 8 || B % ((size_t)w * P))
    return -2;
  std::vector<uint32_t> Pm;
  if (!host_parity(w, k, m, kind, Pm)) return -3;
  DecodePlan pl;
  std::string err;
  if (!make_matrix_decode_plan(k, m, w, Pm, er, e, read_all != 0, pl, err)) return -1;
  if (pl.M > 4) return -2;
  if (w == 16) {
    if (k != 12 || m != 4) return -2;
    if (kind == 2) return mat_fixed2_packet<16, 12, 4, 2>(&pl, blocks, B, P);
    if (kind == 5) return mat_fixed2_packet<16, 12, 4, 5>(&pl, blocks, B, P);
    return -2;
  }
  if (kind == 2) {
    if (k == 10 && m == 4) return mat_fixed2_packet<8, 10, 4, 2>(&pl, blocks, B, P);
    if (k == 6 && m == 3) return mat_fixed2_packet<8, 6, 3, 2>(&pl, blocks, B, P);
  } else if (kind == 5) {
    if (k == 10 && m == 4) return mat_fixed2_packet<8, 10, 4, 5>(&pl, blocks, B, P);
    if (k == 6 && m == 3) return mat_fixed2_packet<8, 6, 3, 5>(&pl, blocks, B, P);
  } else {
    if (k == 10 && m == 4) return mat_fixed2_packet<8, 10, 4, 4>(&pl, blocks, B, P);
  }
  return -2;
}

// Host copy of the parity matrix the library builds (for the tests).
int emu_parity_matrix(int w, int k, int m, int kind, uint32_t* out) {
  std::vector<uint32_t> P;
  if (!host_parity(w, k, m, kind, P)) return -3;
  for (size_t i = 0; i < P.size(); ++i) out[i] = P[i];
  return 0;
}

// Compile-time parity matrix of a registered code (for the tests).
int emu_fixed_parity_matrix(int w, int k, int m, int kind, uint32_t* out) {
  auto copy = [&](const auto& mat, int K, int M) {
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < K; ++j) out[i * K + j] = mat.a[i][j];
    return 0;
  };
  // every (w, k, m) the library compiles matrix kernels for, each kind
#define RSGB_EMU_FIXED(W, K, M)                                                            \
  if (w == W && k == K && m == M) {                                                         \
    if (kind == 1) return copy(ParityMatrix<W, K, M, 1>::value, K, M);                      \
    if (kind == 2) return copy(ParityMatrix<W, K, M, 2>::value, K, M);                      \
    if (kind == 3) return copy(ParityMatrix<W, K, M, 3>::value, K, M);                      \
    if (kind == 5) return copy(ParityMatrix<W, K, M, 5>::value, K, M);                      \
  }
  RSGB_EMU_FIXED(8, 6, 3)
  RSGB_EMU_FIXED(8, 10, 4)
  RSGB_EMU_FIXED(8, 12, 4)
  RSGB_EMU_FIXED(8, 20, 4)
  RSGB_EMU_FIXED(16, 12, 4)
#undef RSGB_EMU_FIXED
  return -2;
}

int emu_poly_encode(int w, int k, int m, uint8_t* blocks, size_t B) {
  return w == 8 ? encode_w<8>(k, m, blocks, B) : (w == 16 ? encode_w<16>(k, m, blocks, B) : -1);
}

int emu_poly_decode(int w, int k, int m, const int* er, int e, int read_all, uint8_t* blocks, size_t B) {
  DecodePlan pl;
  std::string err;
  if (!make_poly_decode_plan(k, m, w, er, e, read_all != 0, pl, err)) return -1;
  if (e == 0) return 0;
  return w == 8 ? decode_w<8>(pl, blocks, B) : decode_w<16>(pl, blocks, B);
}

// The two-column-group compile-time-P encodes (GF(2^8), M <= 4): kinds 1
// and 3 (Vandermonde, generator-matrix form of the polynomial code).
int emu_encode2(int kind, int k, int m, uint8_t* blocks, size_t B) {
  if (kind == 1 && k == 10 && m == 4) return mat_encode2<10, 4, 1>(blocks, B);
  if (kind == 1 && k == 6 && m == 3) return mat_encode2<6, 3, 1>(blocks, B);
  if (kind == 3 && k == 10 && m == 4) return mat_encode2<10, 4, 3>(blocks, B);
  return -2;
}

// The two-column-group decode (GF(2^8), M <= 4).
int emu_poly_decode2(int w, int k, int m, const int* er, int e, int read_all, uint8_t* blocks, size_t B) {
  DecodePlan pl;
  std::string err;
  if (w != 8) return -2;
  if (!make_poly_decode_plan(k, m, w, er, e, read_all != 0, pl, err)) return -1;
  if (e == 0) return 0;
  switch (pl.M) {
    case 1: run_decode2<8, 1>(pl, blocks, B); return 0;
    case 2: run_decode2<8, 2>(pl, blocks, B); return 0;
    case 3: run_decode2<8, 3>(pl, blocks, B); return 0;
    case 4: run_decode2<8, 4>(pl, blocks, B); return 0;
    case 5: run_decode2<8, 5>(pl, blocks, B); return 0;
    case 6: run_decode2<8, 6>(pl, blocks, B); return 0;
  }
  return -2;
}

// Plan introspection for tests: M, read mask, W rows.
int emu_poly_plan(int k, int m, int w, const int* er, int e, int read_all, int* M, uint64_t* read_mask,
                  uint32_t* Wout /* 8x8 */) {
  DecodePlan pl;
  std::string err;
  if (!make_poly_decode_plan(k, m, w, er, e, read_all != 0, pl, err)) return -1;
  *M = pl.M;
  *read_mask = pl.read_mask;
  for (int t = 0; t < 8; ++t)
    for (int j = 0; j < 8; ++j) Wout[t * 8 + j] = pl.W[t][j];
  return 0;
}

// The compile-time generator polynomial coefficients the kernels use.
int emu_genpoly(int w, int m, uint32_t* g) {
  const GenPoly gp = make_genpoly(w, m);
  for (int i = 0; i <= m; ++i) g[i] = gp.c[i];
  return 0;
}

// Transpose round trip and plane semantics for the tests.
int emu_transpose(int w, uint32_t* x) {
  if (w == 8) transpose<8>(x);
  else if (w == 16) transpose<16>(x);
  else return -1;
  return 0;
}

}  // extern "C"
