// Tile geometry of the persistent stripe kernel, host- and device-callable
// (the kernel uses it on the GPU; the host harness checks it on the CPU).
//
// Symbol layout: tile lt of a stripe is bytes [lt*slice, lt*slice + len) of
// every block.
// Packet layout (§2.3): a block is super-packets of W packets of P bytes.
// A unit is G adjacent 32-bit words at the same offset of the W packets of
// one super-packet (U = P / 4G units per super-packet); a block is its
// units super-packet after super-packet, and tile lt is units
// [lt*T, lt*T + len), T = slice / (W*4G).  The tile starts at column col0
// of the super-packet at byte goff; `head` units finish that super-packet
// (0 when the tile starts on a boundary), `whole` complete super-packets
// follow, then len - head - whole*U units of the next.
#pragma once
#include <stdint.h>

#include "gf.hpp"
#include "job.hpp"

namespace rsgb {

struct TileGeom {
  uint64_t goff;
  uint32_t len;
  uint32_t col0;
  uint32_t head;
  uint32_t whole;
};

template <int G>
RS_HD TileGeom tile_geom(const StripeDesc& d, uint32_t lt, uint32_t slice, int w) {
  TileGeom g;
  g.col0 = g.head = g.whole = 0;
  if (d.layout == kLayoutSymbol) {
    g.goff = (uint64_t)lt * slice;
    const uint64_t rem = d.bytes - g.goff;
    g.len = rem < slice ? (uint32_t)rem : slice;
  } else {
    const uint32_t ub = 4u * (uint32_t)G;
    const uint32_t T = slice / ((uint32_t)w * ub);
    const uint32_t U = d.packet_bytes / ub;
    const uint64_t total = d.bytes / ((uint64_t)w * ub);
    const uint64_t u0 = (uint64_t)lt * T;
    const uint64_t rem = total - u0;
    g.len = rem < T ? (uint32_t)rem : T;
    const uint64_t sp = u0 / U;
    g.goff = sp * (uint64_t)w * d.packet_bytes;
    g.col0 = (uint32_t)(u0 - sp * U);
    g.head = g.col0 ? (U - g.col0 < g.len ? U - g.col0 : g.len) : 0u;
    g.whole = (g.len - g.head) / U;
  }
  return g;
}

// Bytes of the whole super-packets one packet tile of `slice` bytes per
// block can touch: a tile of T units starts at a multiple of gcd(T, U)
// inside a super-packet of U units.  When these take at most 3/2 of the
// tile's bytes the slot holds them whole (one bulk copy per block).
inline uint32_t packet_whole_bytes(uint32_t slice, int w, int groups, uint32_t packet_bytes) {
  const uint32_t ub = 4u * (uint32_t)groups;
  const uint32_t T = slice / ((uint32_t)w * ub), U = packet_bytes / ub;
  uint32_t a = T, b = U;
  while (b) {
    const uint32_t r = a % b;
    a = b;
    b = r;
  }
  const uint64_t touched = (uint64_t)(U - a + T - 1u) / U + 1u;
  const uint64_t bytes = touched * (uint64_t)w * packet_bytes;
  return bytes > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)bytes;
}

// The bulk copies that fill a slot for packet tile g: arm(total bytes)
// once, then f(slot offset, offset from the tile's super-packet at goff in
// the block, bytes) per copy.  whole_sp: the super-packets the tile
// touches in one copy; otherwise the rows of the leading partial
// super-packet (W copies), the whole ones after it (one copy) and the rows
// of the trailing partial one (W copies), the slot holding the three parts
// one after the other, each row-major.  Every size is a multiple of 32
// units, so of 128 bytes; every offset is below the slot size.
template <int W, int G, class Arm, class F>
RS_HD void packet_copies(const TileGeom& g, uint32_t P, bool whole_sp, Arm&& arm, F&& f) {
  constexpr uint32_t ub = 4u * (uint32_t)G;
  const uint32_t sp_bytes = (uint32_t)W * P, U = P / ub;
  if (whole_sp) {
    const uint32_t bytes = ((g.col0 + g.len - 1u) / U + 1u) * sp_bytes;
    arm(bytes);
    f(0u, 0u, bytes);
    return;
  }
  arm(g.len * ub * (uint32_t)W);
  const uint32_t tail = g.len - g.head - g.whole * U;
  uint32_t o = 0, b = 0;
  if (g.head) {
    for (int c = 0; c < W; ++c) f(o + (uint32_t)c * g.head * ub, b + (uint32_t)c * P + g.col0 * ub, g.head * ub);
    o += (uint32_t)W * g.head * ub;
    b += sp_bytes;
  }
  if (g.whole) {
    f(o, b, g.whole * sp_bytes);
    o += g.whole * sp_bytes;
    b += g.whole * sp_bytes;
  }
  if (tail) {
    for (int c = 0; c < W; ++c) f(o + (uint32_t)c * tail * ub, b + (uint32_t)c * P, tail * ub);
  }
}

// Where unit `unit` of a packet tile lies: row c of it is at slot byte
// sbase + c*srow and at block byte gbase + c*P.  valid = false for the
// units past a short last tile (they read row 0 of the slot and store
// nothing).
struct UnitPlace {
  uint32_t sbase;
  uint32_t srow;
  uint64_t gbase;
  bool valid;
};

template <int W, int G>
RS_HD UnitPlace packet_unit_place(uint64_t goff, uint32_t len, uint32_t col0, uint32_t head, uint32_t whole,
                                  uint32_t P, bool whole_sp, uint32_t unit) {
  constexpr uint32_t ub = 4u * (uint32_t)G;
  const uint32_t U = P / ub, sp_bytes = (uint32_t)W * P;
  UnitPlace u;
  u.valid = unit < len;
  if (!u.valid) {
    u.sbase = 0;
    u.srow = 0;
    u.gbase = 0;
  } else if (whole_sp) {  // slot = the super-packets from the one at goff on
    const uint32_t v = col0 + unit, j = v / U, col = v - j * U;
    u.sbase = j * sp_bytes + col * ub;
    u.srow = P;
    u.gbase = goff + (uint64_t)j * sp_bytes + (uint64_t)col * ub;
  } else if (unit < head) {  // leading partial super-packet
    u.sbase = unit * ub;
    u.srow = head * ub;
    u.gbase = goff + (uint64_t)(col0 + unit) * ub;
  } else if (unit < head + whole * U) {  // whole super-packets: same layout as the block
    const uint32_t v = unit - head, j = v / U, col = v - j * U;
    u.sbase = (uint32_t)W * ub * head + j * sp_bytes + col * ub;
    u.srow = P;
    u.gbase = goff + (uint64_t)((head ? 1u : 0u) + j) * sp_bytes + (uint64_t)col * ub;
  } else {  // trailing partial super-packet
    const uint32_t before = head + whole * U, v = unit - before;
    u.sbase = (uint32_t)W * ub * before + v * ub;
    u.srow = (len - before) * ub;
    u.gbase = goff + (uint64_t)((head ? 1u : 0u) + whole) * sp_bytes + (uint64_t)v * ub;
  }
  return u;
}

}  // namespace rsgb
